/*
 * pic_adjoint.c -- plain FP64 oracle of the adjoint (reverse-mode gradient) of the collisionless
 * PIC step.  TEST INFRASTRUCTURE ONLY (see pic_oracle.h); shares no code with the GPU library.
 *
 * The paper has no adjoint; this is the differentiation pattern of the task, stated here from the
 * forward model (Sec. 2: gather -> push -> deposit -> field solve, collisions off) and ordinary
 * reverse-mode calculus.  Readings:
 *  - Absorption at the walls is a discrete event.  The forward that is differentiated keeps the
 *    absorption schedule fixed: a "record" run absorbs a particle at the first step its position
 *    leaves [0, N) and stores that step; a "replay" run (used for finite differences) absorbs every
 *    particle at its recorded step whatever its position.  Between its load and its absorption a
 *    particle of a replay run may stand slightly outside [0, N); its CIC weights then extend the
 *    boundary cell linearly (cell clamped to [0, N-1], fraction x - cell outside [0, 1)).
 *  - Observables: J_flux = sum over steps n of dt * sum over electrons alive after step n of
 *    w v_x S(x - (N - 1)), S(d) = max(0, 1 - |d|) (the CIC share of the last interior node, a smooth
 *    stand-in for the electron flux into the right wall), and J_fe = sum_j c_j E_j^2 dx / 2 of the
 *    final node field (c_j = 1/2 at the walls, 1 inside).
 *  - Parameters: the left-wall potential V_L (right wall grounded), which enters every field solve
 *    as the uniform field (V_L - V_R) / (N dx), and the initial electron temperature T_e, which
 *    enters through the loaded velocities v = sqrt(T_e / m) xi with the draws xi fixed.
 *
 * Step n maps (x^n, v^n, E^n) to (x^{n+1}, v^{n+1}, E^{n+1}):
 *   e = (1 - f) E_c + f E_{c+1}          (c, f: CIC cell and fraction of x^n)
 *   v^{n+1} = M v^n + (M + I) h e x_hat  (Boris with uniform B; h = q dt / 2m; M: the rotation)
 *   x^{n+1} = x^n + v_x^{n+1} dt / dx
 *   rho^{n+1} from the particles alive after step n, E^{n+1} = G rho^{n+1} + (V_L - V_R)/(N dx).
 * The reverse sweep carries lambda = dJ/d(x, v) per particle and mu = dJ/dE per node backwards:
 *   rho_bar = G^T mu^{n+1}; dJ/dV_L += sum_j mu^{n+1}_j / (N dx)
 *   per particle alive after step n: lambda_x += q w (rho_bar_{c'+1}/vol_{c'+1} - rho_bar_{c'}/vol_{c'})
 *     (+ the J_flux terms at x^{n+1}, v^{n+1} for electrons), lambda_vx += lambda_x dt / dx,
 *     e_bar = h [(M + I)^T lambda_v]_x, lambda_x += e_bar (E^n_{c+1} - E^n_c),
 *     lambda_v = M^T lambda_v, mu^n_c += e_bar (1 - f), mu^n_{c+1} += e_bar f
 * and finally dJ/dT_e = sum over electrons lambda_v . v^0 / (2 T_e).
 * G^T: with psi = D^T mu (D: the node-field differences as functions of the interior potential),
 * rho_bar_int = dx^2 A^{-1} psi (A = tridiag(-1, 2, -1) is symmetric: the same Thomas solve),
 * rho_bar_0 = -mu_0 dx / 2 and rho_bar_N = mu_N dx / 2 (the Gauss terms at the walls).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include "pic_oracle.h"

typedef struct {
  int32_t N;
  double dx;
  size_t n0, np;      /* electrons are particles [0, n0), ions [n0, np) */
  double q[2], w[2], h[2], qm[2];
  double Bv[3];
  double M[2][3][3];  /* Boris rotation of each species: v' = M v for E = 0 */
} adj_model;

static void adj_model_init(const orc_config* c, adj_model* m) {
  memset(m, 0, sizeof(*m));
  m->N = c->ncells;
  m->dx = c->L / (double)c->ncells;
  m->n0 = (size_t)c->ppc[0] * (size_t)c->ncells;
  m->np = m->n0 + (size_t)c->ppc[1] * (size_t)c->ncells;
  const double th = c->B_angle_deg * 3.14159265358979323846 / 180.0;
  m->Bv[0] = c->B * cos(th);
  m->Bv[1] = c->B * sin(th);
  m->Bv[2] = 0.0;
  for (int s = 0; s < 2; ++s) {
    m->q[s] = c->charge[s];
    m->w[s] = m->dx / (double)c->ppc[s];
    m->qm[s] = c->charge[s] / c->mass[s];
    m->h[s] = 0.5 * m->qm[s] * c->dt;
    const double zero[3] = {0.0, 0.0, 0.0};
    for (int k = 0; k < 3; ++k) { /* column k: the rotation of the unit vector e_k */
      double v[3] = {0.0, 0.0, 0.0};
      v[k] = 1.0;
      orc_boris(m->qm[s], c->dt, zero, m->Bv, v);
      for (int i = 0; i < 3; ++i) m->M[s][i][k] = v[i];
    }
  }
}

/* CIC cell and fraction, the cell clamped to [0, N-1] (linear extension outside [0, N)). */
static void cic(int32_t N, double x, int32_t* c, double* f) {
  double fl = floor(x);
  int32_t k = (int32_t)fl;
  if (fl < 0.0) k = 0;
  if (fl > (double)(N - 1)) k = N - 1;
  *c = k;
  *f = x - (double)k;
}

static double vol(const adj_model* m, int32_t j) { return (j == 0 || j == m->N) ? 0.5 * m->dx : m->dx; }

/* Node charge density of the particles with absorb[p] > after (alive after that step). */
static void density(const adj_model* m, const double* x, const int32_t* absorb, int32_t after, double* rho) {
  memset(rho, 0, sizeof(double) * (size_t)(m->N + 1));
  for (size_t p = 0; p < m->np; ++p) {
    if (absorb[p] <= after) continue;
    const int s = p < m->n0 ? 0 : 1;
    int32_t c;
    double f;
    cic(m->N, x[p], &c, &f);
    rho[c] += m->q[s] * m->w[s] * (1.0 - f);
    rho[c + 1] += m->q[s] * m->w[s] * f;
  }
  for (int32_t j = 0; j <= m->N; ++j) rho[j] /= vol(m, j);
}

static void field(const orc_config* c, const adj_model* m, const double* rho, double* phi, double* E) {
  orc_poisson_thomas(m->N, m->dx, rho, c->V_left, c->V_right, phi);
  orc_efield(m->N, m->dx, phi, rho, E);
}

void orc_field_apply(int32_t N, double dx, const double* rho, double* E) {
  double* phi = (double*)malloc(sizeof(double) * (size_t)(N + 1));
  orc_poisson_thomas(N, dx, rho, 0.0, 0.0, phi);
  orc_efield(N, dx, phi, rho, E);
  free(phi);
}

void orc_field_adjoint(int32_t N, double dx, const double* mu, double* rho_bar) {
  double* psi = (double*)calloc((size_t)(N + 1), sizeof(double));
  double* chi = (double*)malloc(sizeof(double) * (size_t)(N + 1));
  /* psi = D^T mu over the interior potentials phi_1 .. phi_{N-1} */
  for (int32_t k = 1; k <= N - 1; ++k) {
    double a = 0.0;
    if (k + 1 <= N - 1) a += mu[k + 1] / (2.0 * dx); /* E_{k+1} = (phi_k - phi_{k+2}) / 2dx */
    if (k - 1 >= 1) a -= mu[k - 1] / (2.0 * dx);     /* E_{k-1} = (phi_{k-2} - phi_k) / 2dx */
    if (k == 1) a -= mu[0] / dx;                     /* E_0 = (phi_0 - phi_1) / dx - ...   */
    if (k == N - 1) a += mu[N] / dx;                 /* E_N = (phi_{N-1} - phi_N) / dx + ... */
    psi[k] = a / (dx * dx);                          /* the Thomas solve multiplies by dx^2 */
  }
  orc_poisson_thomas(N, dx, psi, 0.0, 0.0, chi); /* chi = A^{-1} psi (A symmetric) */
  for (int32_t k = 1; k <= N - 1; ++k) rho_bar[k] = dx * dx * chi[k];
  rho_bar[0] = -mu[0] * dx / 2.0;
  rho_bar[N] = mu[N] * dx / 2.0;
  free(psi);
  free(chi);
}

/* One push of particle p with the node field E (field_mode as the configuration says). */
static void push(const orc_config* c, const adj_model* m, int s, const double* E, double* x, double v[3]) {
  double Ex = 0.0;
  if (c->field_mode == ORC_FIELD_SELF) {
    int32_t k;
    double f;
    cic(m->N, *x, &k, &f);
    Ex = (1.0 - f) * E[k] + f * E[k + 1];
  } else if (c->field_mode == ORC_FIELD_EXTERNAL) {
    Ex = c->E_ext;
  }
  const double Ev[3] = {Ex, 0.0, 0.0};
  orc_boris(m->qm[s], c->dt, Ev, m->Bv, v);
  *x += v[0] * c->dt / m->dx;
}

static double flux_share(const adj_model* m, double x) {
  const double d = fabs(x - (double)(m->N - 1));
  return d < 1.0 ? 1.0 - d : 0.0;
}

static double field_energy(const adj_model* m, const double* E) {
  double fe = 0.0;
  for (int32_t j = 0; j <= m->N; ++j) fe += ((j == 0 || j == m->N) ? 0.5 : 1.0) * 0.5 * E[j] * E[j] * m->dx;
  return fe;
}

static int valid_adj(const orc_config* c, int32_t steps) {
  if (!c || steps < 0 || c->ncells < 2 || c->ppc[0] < 1 || c->ppc[1] < 1 || !(c->L > 0) || !(c->dt > 0)) return 0;
  if (c->coll_mask != 0 || c->source_mode != ORC_SOURCE_NONE || !(c->T[0] > 0)) return 0;
  return 1;
}

/* The frozen-schedule forward.  Optionally keeps the trajectory: X[(T+1) np], V[(T+1) 3 np],
 * EN[(T+1)(N+1)] (E^n: the field the push of step n uses; E^T: the final field). */
static int forward(const orc_config* c, int32_t steps, int replay, int32_t* absorb, double J[2], double* X,
                   double* V, double* EN) {
  adj_model m;
  adj_model_init(c, &m);
  const int32_t N = m.N;
  double* x = (double*)malloc(sizeof(double) * m.np);
  double* v = (double*)malloc(sizeof(double) * 3 * m.np);
  double* rho = (double*)malloc(sizeof(double) * (size_t)(N + 1));
  double* phi = (double*)malloc(sizeof(double) * (size_t)(N + 1));
  double* E = (double*)malloc(sizeof(double) * (size_t)(N + 1));
  if (!x || !v || !rho || !phi || !E) {
    free(x), free(v), free(rho), free(phi), free(E);
    return ORC_ENOMEM;
  }
  for (size_t p = 0; p < m.np; ++p) {
    const int s = p < m.n0 ? 0 : 1;
    uint64_t id;
    orc_load_particle(c, s, s ? p - m.n0 : p, &x[p], &v[3 * p], &id);
    if (!replay) absorb[p] = ORC_ADJ_NEVER;
  }
  density(&m, x, absorb, -1, rho);
  field(c, &m, rho, phi, E);
  double jf = 0.0;
  for (int32_t n = 0; n < steps; ++n) {
    if (X) {
      memcpy(X + (size_t)n * m.np, x, sizeof(double) * m.np);
      memcpy(V + (size_t)n * 3 * m.np, v, sizeof(double) * 3 * m.np);
      memcpy(EN + (size_t)n * (size_t)(N + 1), E, sizeof(double) * (size_t)(N + 1));
    }
    for (size_t p = 0; p < m.np; ++p) {
      if (absorb[p] < n) continue; /* absorbed in an earlier step */
      const int s = p < m.n0 ? 0 : 1;
      if (!(c->frozen_mask & (1u << s))) push(c, &m, s, E, &x[p], &v[3 * p]);
      if (!replay && (x[p] < 0.0 || x[p] >= (double)N)) absorb[p] = n;
    }
    for (size_t p = 0; p < m.n0; ++p)
      if (absorb[p] > n) jf += c->dt * m.w[0] * v[3 * p] * flux_share(&m, x[p]);
    density(&m, x, absorb, n, rho);
    field(c, &m, rho, phi, E);
  }
  if (X) {
    memcpy(X + (size_t)steps * m.np, x, sizeof(double) * m.np);
    memcpy(V + (size_t)steps * 3 * m.np, v, sizeof(double) * 3 * m.np);
    memcpy(EN + (size_t)steps * (size_t)(N + 1), E, sizeof(double) * (size_t)(N + 1));
  }
  J[0] = jf;
  J[1] = field_energy(&m, E);
  free(x), free(v), free(rho), free(phi), free(E);
  return ORC_OK;
}

size_t orc_adj_particles(const orc_config* c) {
  return (size_t)c->ppc[0] * (size_t)c->ncells + (size_t)c->ppc[1] * (size_t)c->ncells;
}

int orc_adj_forward(const orc_config* c, int32_t steps, int replay, int32_t* absorb, double J[2]) {
  if (!valid_adj(c, steps) || !absorb || !J) return ORC_EINVAL;
  return forward(c, steps, replay, absorb, J, NULL, NULL, NULL);
}

/* The reverse sweep over a stored trajectory (X, V, EN as forward() keeps it, absorb the schedule):
 * grad = d(wt[0] J_flux + wt[1] J_fe) / d(V_left, T[0]). */
static int reverse(const orc_config* c, int32_t steps, const double wt[2], const double* X, const double* V,
                   const double* EN, const int32_t* absorb, double grad[2]) {
  adj_model m;
  adj_model_init(c, &m);
  const int32_t N = m.N;
  const size_t np = m.np, nn = (size_t)(N + 1);
  double* lx = (double*)calloc(np, sizeof(double));
  double* lv = (double*)calloc(3 * np, sizeof(double));
  double* mu = (double*)malloc(sizeof(double) * nn);
  double* mu_next = (double*)malloc(sizeof(double) * nn);
  double* rb = (double*)malloc(sizeof(double) * nn);
  if (!lx || !lv || !mu || !mu_next || !rb) {
    free(lx), free(lv), free(mu), free(mu_next), free(rb);
    return ORC_ENOMEM;
  }
  double gV = 0.0;
  /* dJ/dE^T: the final field energy */
  const double* ET = EN + (size_t)steps * nn;
  for (int32_t j = 0; j <= N; ++j) mu[j] = wt[1] * ((j == 0 || j == N) ? 0.5 : 1.0) * ET[j] * m.dx;
  for (int32_t n = steps - 1; n >= 0; --n) {
    /* E^{n+1} = G rho^{n+1} + (V_L - V_R) / (N dx) */
    for (int32_t j = 0; j <= N; ++j) gV += mu[j] / ((double)N * m.dx);
    orc_field_adjoint(N, m.dx, mu, rb);
    const double* x1 = X + (size_t)(n + 1) * np;
    const double* v1 = V + (size_t)(n + 1) * 3 * np;
    const double* x0 = X + (size_t)n * np;
    const double* En = EN + (size_t)n * nn;
    memset(mu_next, 0, sizeof(double) * nn);
    for (size_t p = 0; p < np; ++p) {
      if (absorb[p] <= n) continue; /* not alive after step n: nothing depends on its state */
      const int s = p < m.n0 ? 0 : 1;
      /* deposit of x^{n+1} */
      int32_t k1;
      double f1;
      cic(N, x1[p], &k1, &f1);
      lx[p] += m.q[s] * m.w[s] * (rb[k1 + 1] / vol(&m, k1 + 1) - rb[k1] / vol(&m, k1));
      /* J_flux at step n */
      if (s == 0) {
        const double d = x1[p] - (double)(N - 1);
        if (fabs(d) < 1.0) {
          lx[p] += wt[0] * c->dt * m.w[0] * v1[3 * p] * (d > 0.0 ? -1.0 : (d < 0.0 ? 1.0 : 0.0));
          lv[3 * p] += wt[0] * c->dt * m.w[0] * (1.0 - fabs(d));
        }
      }
      if (c->frozen_mask & (1u << s)) continue; /* not pushed: x^{n+1} = x^n, v^{n+1} = v^n */
      /* x^{n+1} = x^n + v_x^{n+1} dt / dx */
      lv[3 * p] += lx[p] * c->dt / m.dx;
      /* v^{n+1} = M v^n + (M + I) h e */
      double* L = &lv[3 * p];
      double ebar = 0.0;
      if (c->field_mode == ORC_FIELD_SELF) {
        for (int i = 0; i < 3; ++i) ebar += (m.M[s][i][0] + (i == 0 ? 1.0 : 0.0)) * L[i];
        ebar *= m.h[s];
        int32_t k0;
        double f0;
        cic(N, x0[p], &k0, &f0);
        lx[p] += ebar * (En[k0 + 1] - En[k0]);
        mu_next[k0] += ebar * (1.0 - f0);
        mu_next[k0 + 1] += ebar * f0;
      }
      double Lt[3];
      for (int k = 0; k < 3; ++k) Lt[k] = m.M[s][0][k] * L[0] + m.M[s][1][k] * L[1] + m.M[s][2][k] * L[2];
      L[0] = Lt[0], L[1] = Lt[1], L[2] = Lt[2];
    }
    memcpy(mu, mu_next, sizeof(double) * nn);
  }
  /* E^0 = G rho^0 + bias; rho^0 does not depend on the parameters */
  for (int32_t j = 0; j <= N; ++j) gV += mu[j] / ((double)N * m.dx);
  double gT = 0.0;
  for (size_t p = 0; p < m.n0; ++p)
    for (int k = 0; k < 3; ++k) gT += lv[3 * p + k] * V[3 * p + k];
  grad[0] = gV;
  grad[1] = gT / (2.0 * c->T[0]);
  free(lx), free(lv), free(mu), free(mu_next), free(rb);
  return ORC_OK;
}

int orc_adj_gradient(const orc_config* c, int32_t steps, const double wt[2], double grad[2], double J[2],
                     int32_t* absorb) {
  if (!valid_adj(c, steps) || !wt || !grad || !J || !absorb) return ORC_EINVAL;
  adj_model m;
  adj_model_init(c, &m);
  const size_t np = m.np, nn = (size_t)(m.N + 1);
  double* X = (double*)malloc(sizeof(double) * (size_t)(steps + 1) * np);
  double* V = (double*)malloc(sizeof(double) * (size_t)(steps + 1) * 3 * np);
  double* EN = (double*)malloc(sizeof(double) * (size_t)(steps + 1) * nn);
  int rc = ORC_ENOMEM;
  if (X && V && EN) rc = forward(c, steps, 0, absorb, J, X, V, EN);
  if (rc == ORC_OK) rc = reverse(c, steps, wt, X, V, EN, absorb, grad);
  free(X), free(V), free(EN);
  return rc;
}

int orc_adj_trajectory(const orc_config* c, int32_t steps, double* X, double* V, double* EN, int32_t* absorb,
                       double J[2]) {
  if (!valid_adj(c, steps) || !X || !V || !EN || !absorb || !J) return ORC_EINVAL;
  return forward(c, steps, 0, absorb, J, X, V, EN);
}

int orc_adj_gradient_from_tape(const orc_config* c, int32_t steps, const double wt[2], const double* X,
                               const double* V, const double* EN, const int32_t* absorb, double grad[2]) {
  if (!valid_adj(c, steps) || !wt || !grad || !X || !V || !EN || !absorb) return ORC_EINVAL;
  return reverse(c, steps, wt, X, V, EN, absorb, grad);
}
