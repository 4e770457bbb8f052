// api_adjoint.cu -- the adjoint entry points of include/pic.h (pic_adj_*): gradients of the wall
// electron flux and of the final field energy of a collisionless run with respect to the left-wall
// potential and the initial electron temperature, by a discrete adjoint with step checkpointing.
//
// Forward (pic_adj_forward): load, then `steps` FP32 steps (k_adj_push, one FP64 field solve per
// step from the signed fixed-point deposits).  A recording run stores the absorption schedule, the
// particle state every `checkpoint_every` steps and the FP64 node field of every step (N + 1
// values a step: small next to the particles).  A replaying run reuses the schedule and writes no
// tape (finite differences of the same frozen-schedule map).
// Reverse (pic_adj_gradient): for each segment of checkpoint_every steps, last segment first, the
// segment's particle states are recomputed from its checkpoint with the stored fields (the same
// kernel and inputs as the recording run: bit-identical), then the steps are reversed one by one.
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "api_internal.h"

using namespace picx;

struct pic_adj {
  pic_config cfg;
  int T = 0, K = 0, nseg = 0, N = 0;
  unsigned long long n0 = 0, np = 0;
  cudaStream_t st = nullptr;
  void* ws = nullptr;
  size_t ws_bytes = 0;
  bool owns_ws = false;
  AdjState cur;
  unsigned long long* id = nullptr;
  int* absorb = nullptr;
  std::vector<AdjState> ckpt, tape;
  double *lx = nullptr, *lvx = nullptr, *lvy = nullptr, *lvz = nullptr;
  unsigned long long* R[2] = {nullptr, nullptr};
  double *rho = nullptr, *phi = nullptr, *Etape = nullptr, *Escr[2] = {nullptr, nullptr};
  double *mu = nullptr, *mu_next = nullptr, *rhs = nullptr, *chi = nullptr;
  double* gV = nullptr;
  unsigned long long* jflux = nullptr;
  double* partial = nullptr;
  int tblocks = 304, max_grid = 152 * 8;
  bool recorded = false;
  double rec_VL = 0.0, rec_Te = 0.0;
  float ms_fwd = 0.f, ms_rev = 0.f;
};

namespace {

#define CKA(x)                                \
  do {                                        \
    cudaError_t e__ = (x);                    \
    if (e__ != cudaSuccess) return PIC_ECUDA; \
  } while (0)

bool adj_valid(const pic_config* c, int32_t steps, int32_t K) {
  if (!valid(c)) return false;
  if (c->coll_mask != 0u || c->source_mode != PIC_SOURCE_NONE || !(c->T[0] > 0)) return false;
  if (c->neutrals || c->smooth_passes) return false;  // the adjoint differentiates the plain step
  if (steps < 1 || K < 1 || K > steps) return false;
  const double np = (double)c->ncells * ((double)c->ppc[0] + (double)c->ppc[1]);
  return np < 2147483648.0;
}

struct Carve {
  char* base;
  size_t off = 0;
  template <class T>
  T* take(size_t count) {
    off = (off + 255) & ~size_t(255);
    T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
    off += sizeof(T) * count;
    return p;
  }
};

AdjState take_state(Carve& cv, size_t n) {
  AdjState s;
  s.cell = cv.take<int>(n);
  s.frac = cv.take<float>(n);
  s.vx = cv.take<float>(n);
  s.vy = cv.take<float>(n);
  s.vz = cv.take<float>(n);
  return s;
}

void layout(pic_adj* a, char* base, size_t* total) {
  Carve cv{base};
  const size_t np = (size_t)a->np, nn = (size_t)a->N + 1;
  a->cur = take_state(cv, np);
  a->id = cv.take<unsigned long long>(np);
  a->absorb = cv.take<int>(np);
  a->ckpt.resize(a->nseg);
  for (int k = 0; k < a->nseg; ++k) a->ckpt[k] = take_state(cv, np);
  a->tape.resize(a->K + 1);
  for (int k = 0; k <= a->K; ++k) a->tape[k] = take_state(cv, np);
  a->lx = cv.take<double>(np);
  a->lvx = cv.take<double>(np);
  a->lvy = cv.take<double>(np);
  a->lvz = cv.take<double>(np);
  for (int s = 0; s < 2; ++s) a->R[s] = cv.take<unsigned long long>(nn);
  a->rho = cv.take<double>(nn);
  a->phi = cv.take<double>(nn);
  a->Etape = cv.take<double>(nn * (size_t)(a->T + 1));
  for (int k = 0; k < 2; ++k) a->Escr[k] = cv.take<double>(nn);
  a->mu = cv.take<double>(nn);
  a->mu_next = cv.take<double>(nn);
  a->rhs = cv.take<double>(nn);
  a->chi = cv.take<double>(nn);
  a->gV = cv.take<double>(1);
  a->jflux = cv.take<unsigned long long>(1);
  a->partial = cv.take<double>((size_t)a->tblocks);
  *total = cv.off + 256;
}

void init_dims(pic_adj* a, const pic_config* c, int32_t steps, int32_t K) {
  a->cfg = *c;
  a->T = steps;
  a->K = K;
  a->nseg = (steps + K - 1) / K;
  a->N = c->ncells;
  a->n0 = (unsigned long long)c->ppc[0] * (unsigned long long)c->ncells;
  a->np = a->n0 + (unsigned long long)c->ppc[1] * (unsigned long long)c->ncells;
}

// Physics constants of a parameter point (the single-run derivation of the library).
Phys physics(const pic_adj* a, double VL, double Te, pic_config* out) {
  pic_config c = a->cfg;
  c.V_left = VL;
  c.T[0] = Te;
  pic_handle tmp;
  tmp.cfg = c;
  tmp.N = c.ncells;
  derive(&tmp);
  *out = c;
  return tmp.ph;
}

PoissonParams field_from_R(const pic_adj* a, const pic_config& c, double* E) {
  PoissonParams F;
  std::memset(&F, 0, sizeof(F));
  const double dx = c.L / c.ncells;
  for (int s = 0; s < 2; ++s) {
    F.R[s] = reinterpret_cast<long long*>(a->R[s]);
    F.qw[s] = c.charge[s] * (dx / c.ppc[s]);
  }
  F.mode = 3;
  F.zero_R = 1;  // the next push deposits into R again
  F.N = c.ncells;
  F.dx = dx;
  F.inv_dx = 1.0 / dx;
  F.V_L = c.V_left;
  F.V_R = c.V_right;
  F.rho = a->rho;
  F.phi = a->phi;
  F.E = E;
  return F;
}

int copy_state(const pic_adj* a, const AdjState& dst, const AdjState& src) {
  const size_t n = (size_t)a->np;
  CKA(cudaMemcpyAsync(dst.cell, src.cell, 4 * n, cudaMemcpyDeviceToDevice, a->st));
  CKA(cudaMemcpyAsync(dst.frac, src.frac, 4 * n, cudaMemcpyDeviceToDevice, a->st));
  CKA(cudaMemcpyAsync(dst.vx, src.vx, 4 * n, cudaMemcpyDeviceToDevice, a->st));
  CKA(cudaMemcpyAsync(dst.vy, src.vy, 4 * n, cudaMemcpyDeviceToDevice, a->st));
  CKA(cudaMemcpyAsync(dst.vz, src.vz, 4 * n, cudaMemcpyDeviceToDevice, a->st));
  return PIC_OK;
}

AdjStep step_params(const pic_adj* a, const Phys& ph, const pic_config& c) {
  AdjStep S;
  std::memset(&S, 0, sizeof(S));
  S.absorb = a->absorb;
  for (int s = 0; s < 2; ++s) {
    S.R[s] = a->R[s];
    S.qmdt2[s] = ph.sp[s].qmdt2;
    for (int i = 0; i < 3; ++i) {
      S.t[s][i] = ph.sp[s].t[i];
      S.s[s][i] = ph.sp[s].s[i];
    }
  }
  S.jflux_fx = a->jflux;
  S.n0 = a->n0;
  S.np = a->np;
  S.N = a->N;
  S.field_mode = c.field_mode;
  S.frozen_mask = c.frozen_mask;
  S.has_B = ph.has_B;
  S.dtdx = ph.dtdx;
  S.E_ext = ph.E_ext;
  S.flux_dtw = c.dt * ((c.L / c.ncells) / c.ppc[0]);
  return S;
}

double field_energy_host(const std::vector<double>& E, int N, double dx) {
  double fe = 0.0;
  for (int j = 0; j <= N; ++j) fe += ((j == 0 || j == N) ? 0.5 : 1.0) * 0.5 * E[j] * E[j] * dx;
  return fe;
}

}  // namespace

extern "C" {

int pic_adj_workspace_size(const pic_config* cfg, int32_t steps, int32_t checkpoint_every, size_t* bytes) {
  PIC_ENTRY_TRY
  if (!bytes || !adj_valid(cfg, steps, checkpoint_every)) return PIC_EINVAL;
  pic_adj tmp;
  init_dims(&tmp, cfg, steps, checkpoint_every);
  layout(&tmp, nullptr, bytes);
  return PIC_OK;
  PIC_ENTRY_CATCH
}

int pic_adj_init(const pic_config* cfg, int32_t steps, int32_t checkpoint_every, void* workspace,
                 size_t workspace_bytes, void* cuda_stream, pic_adj** out) {
  PIC_ENTRY_TRY
  if (!out) return PIC_EINVAL;
  *out = nullptr;
  if (!adj_valid(cfg, steps, checkpoint_every)) return PIC_EINVAL;
  if (workspace && (reinterpret_cast<uintptr_t>(workspace) & 255u)) return PIC_EINVAL;
  pic_adj* a = new (std::nothrow) pic_adj();
  if (!a) return PIC_ENOMEM;
  try {
    init_dims(a, cfg, steps, checkpoint_every);
    a->st = static_cast<cudaStream_t>(cuda_stream);
    size_t need = 0;
    layout(a, nullptr, &need);
    if (workspace) {
      if (workspace_bytes < need) {
        delete a;
        return PIC_ENOMEM;
      }
      a->ws = workspace;
    } else {
      if (cudaMalloc(&a->ws, need) != cudaSuccess) {
        delete a;
        return PIC_ENOMEM;
      }
      a->owns_ws = true;
    }
    a->ws_bytes = need;
    layout(a, static_cast<char*>(a->ws), &need);
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms > 0) a->max_grid = sms * 8;
    *out = a;
    return PIC_OK;
  } catch (...) {  // a host allocation or thread failed part way: release what was taken
    pic_adj_free(a);
    *out = nullptr;
    return PIC_ENOMEM;
  }
  PIC_ENTRY_CATCH
}

int pic_adj_forward(pic_adj* a, double V_left, double T_e, int32_t replay, double J[2]) {
  PIC_ENTRY_TRY
  if (!a || !J || !(T_e > 0) || !std::isfinite(V_left)) return PIC_EINVAL;
  if (replay && !a->recorded) return PIC_EINVAL;
  pic_config c;
  const Phys ph = physics(a, V_left, T_e, &c);
  const int mode = replay ? 1 : 0;
  const size_t nn = (size_t)a->N + 1;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaEventRecord(e0, a->st);
  if (!replay) a->recorded = false;  // the tape is being rewritten
  // load
  StepParams32 L;
  std::memset(&L, 0, sizeof(L));
  L.sp[0] = Species32{a->cur.cell, a->cur.frac, a->cur.vx, a->cur.vy, a->cur.vz, a->id};
  L.sp[1] = Species32{a->cur.cell + a->n0, a->cur.frac + a->n0, a->cur.vx + a->n0, a->cur.vy + a->n0,
                      a->cur.vz + a->n0, a->id + a->n0};
  L.ph = ph;
  const unsigned long long n[2] = {a->n0, a->np - a->n0};
  CKA(launch_load32(L, n, c.load_profile, c.ppc[0], c.ppc[1], c.profile_scale, c.profile_mode, a->st));
  if (!replay) CKA(launch_adj_fill(a->absorb, a->np, 0x7FFFFFFF, a->st));
  CKA(cudaMemsetAsync(a->jflux, 0, sizeof(unsigned long long), a->st));
  for (int s = 0; s < 2; ++s) CKA(cudaMemsetAsync(a->R[s], 0, sizeof(unsigned long long) * nn, a->st));
  CKA(launch_adj_deposit0(a->cur, a->n0, a->np, a->R[0], a->R[1], a->max_grid, a->st));
  double* Ein = replay ? a->Escr[0] : a->Etape;
  CKA(launch_field(field_from_R(a, c, Ein), a->st));
  if (!replay) {
    const int rc = copy_state(a, a->ckpt[0], a->cur);
    if (rc != PIC_OK) return rc;
  }
  AdjStep S = step_params(a, ph, c);
  S.src = S.dst = a->cur;
  S.mode = mode;
  for (int k = 0; k < a->T; ++k) {
    if (!replay && k > 0 && k % a->K == 0) {
      const int rc = copy_state(a, a->ckpt[k / a->K], a->cur);
      if (rc != PIC_OK) return rc;
    }
    double* Eout = replay ? a->Escr[(k + 1) & 1] : a->Etape + (size_t)(k + 1) * nn;
    S.E = Ein;
    S.step = k;
    CKA(launch_adj_push(S, a->max_grid, a->st));
    CKA(launch_field(field_from_R(a, c, Eout), a->st));
    Ein = Eout;
  }
  cudaEventRecord(e1, a->st);
  unsigned long long jf = 0;
  std::vector<double> E(nn);
  CKA(cudaMemcpyAsync(&jf, a->jflux, sizeof(jf), cudaMemcpyDeviceToHost, a->st));
  CKA(cudaMemcpyAsync(E.data(), Ein, sizeof(double) * nn, cudaMemcpyDeviceToHost, a->st));
  CKA(cudaStreamSynchronize(a->st));
  cudaEventElapsedTime(&a->ms_fwd, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  J[0] = (double)(long long)jf * (1.0 / 1099511627776.0);
  J[1] = field_energy_host(E, a->N, c.L / c.ncells);
  if (!replay) {
    a->recorded = true;
    a->rec_VL = V_left;
    a->rec_Te = T_e;
  }
  return PIC_OK;
  PIC_ENTRY_CATCH
}

int pic_adj_gradient(pic_adj* a, const double w[2], double grad[2]) {
  PIC_ENTRY_TRY
  if (!a || !w || !grad || !a->recorded) return PIC_EINVAL;
  pic_config c;
  const Phys ph = physics(a, a->rec_VL, a->rec_Te, &c);
  const int N = a->N;
  const size_t nn = (size_t)N + 1, np = (size_t)a->np;
  const double dx = c.L / c.ncells;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaEventRecord(e0, a->st);
  // lambda = 0, mu^T = w_fe dJ_fe/dE^T, dJ/dV_L = 0
  CKA(cudaMemsetAsync(a->lx, 0, 8 * np, a->st));
  CKA(cudaMemsetAsync(a->lvx, 0, 8 * np, a->st));
  CKA(cudaMemsetAsync(a->lvy, 0, 8 * np, a->st));
  CKA(cudaMemsetAsync(a->lvz, 0, 8 * np, a->st));
  CKA(cudaMemsetAsync(a->gV, 0, sizeof(double), a->st));
  std::vector<double> ET(nn);
  CKA(cudaMemcpyAsync(ET.data(), a->Etape + (size_t)a->T * nn, sizeof(double) * nn, cudaMemcpyDeviceToHost, a->st));
  CKA(cudaStreamSynchronize(a->st));
  for (int j = 0; j <= N; ++j) ET[j] = w[1] * ((j == 0 || j == N) ? 0.5 : 1.0) * ET[j] * dx;
  double* mu = a->mu;
  double* mu_next = a->mu_next;
  CKA(cudaMemcpyAsync(mu, ET.data(), sizeof(double) * nn, cudaMemcpyHostToDevice, a->st));
  // reverse-sweep constants
  AdjRev R;
  std::memset(&R, 0, sizeof(R));
  R.absorb = a->absorb;
  R.chi = a->chi;
  R.lx = a->lx;
  R.lvx = a->lvx;
  R.lvy = a->lvy;
  R.lvz = a->lvz;
  R.n0 = a->n0;
  R.np = a->np;
  R.N = N;
  R.field_mode = c.field_mode;
  R.frozen_mask = c.frozen_mask;
  R.dx = dx;
  R.dtdx = c.dt / dx;
  for (int s = 0; s < 2; ++s) {
    R.qw[s] = c.charge[s] * (dx / c.ppc[s]);
    R.h[s] = ph.sp[s].qmdt2_d;
    // Boris rotation of species s for E = 0: v' = v + (v + v x t) x s, column by column
    const double* t = ph.sp[s].t_d;
    const double* q = ph.sp[s].s_d;
    for (int k = 0; k < 3; ++k) {
      double v[3] = {0.0, 0.0, 0.0};
      v[k] = 1.0;
      const double p[3] = {v[0] + (v[1] * t[2] - v[2] * t[1]), v[1] + (v[2] * t[0] - v[0] * t[2]),
                           v[2] + (v[0] * t[1] - v[1] * t[0])};
      const double r[3] = {v[0] + (p[1] * q[2] - p[2] * q[1]), v[1] + (p[2] * q[0] - p[0] * q[2]),
                           v[2] + (p[0] * q[1] - p[1] * q[0])};
      for (int i = 0; i < 3; ++i) R.M[s][3 * i + k] = r[i];
    }
  }
  R.flux_dtw = w[0] * c.dt * (dx / c.ppc[0]);
  AdjStep S = step_params(a, ph, c);
  S.mode = 2;
  PoissonParams F;  // chi = A^{-1} psi: the Green's-function solve with grounded walls
  std::memset(&F, 0, sizeof(F));
  F.mode = 2;
  F.N = N;
  F.dx = dx;
  F.inv_dx = 1.0 / dx;
  F.rho_in = a->rhs;
  F.phi = a->chi;
  for (int seg = a->nseg - 1; seg >= 0; --seg) {
    const int n0 = seg * a->K, n1 = std::min(a->T, n0 + a->K);
    int rc = copy_state(a, a->tape[0], a->ckpt[seg]);
    if (rc != PIC_OK) return rc;
    for (int k = n0; k < n1; ++k) {  // recompute the segment's states
      S.src = a->tape[k - n0];
      S.dst = a->tape[k + 1 - n0];
      S.E = a->Etape + (size_t)k * nn;
      S.step = k;
      CKA(launch_adj_push(S, a->max_grid, a->st));
    }
    for (int k = n1 - 1; k >= n0; --k) {
      CKA(launch_adj_field_t(mu, a->rhs, N, dx, a->gV, 1, mu_next, a->st));
      CKA(launch_field(F, a->st));
      R.s0 = a->tape[k - n0];
      R.s1 = a->tape[k + 1 - n0];
      R.E = a->Etape + (size_t)k * nn;
      R.mu = mu;
      R.mu_next = mu_next;
      R.step = k;
      CKA(launch_adj_reverse(R, a->max_grid, a->st));
      std::swap(mu, mu_next);
    }
  }
  CKA(launch_adj_field_t(mu, nullptr, N, dx, a->gV, 0, nullptr, a->st));  // E^0's bias term
  CKA(launch_adj_tgrad(R, a->ckpt[0], a->partial, a->tblocks, a->st));
  cudaEventRecord(e1, a->st);
  double gV = 0.0;
  std::vector<double> part(a->tblocks);
  CKA(cudaMemcpyAsync(&gV, a->gV, sizeof(double), cudaMemcpyDeviceToHost, a->st));
  CKA(cudaMemcpyAsync(part.data(), a->partial, sizeof(double) * a->tblocks, cudaMemcpyDeviceToHost, a->st));
  CKA(cudaStreamSynchronize(a->st));
  cudaEventElapsedTime(&a->ms_rev, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  double gT = 0.0;
  for (double v : part) gT += v;
  grad[0] = gV;
  grad[1] = gT / (2.0 * a->rec_Te);
  return PIC_OK;
  PIC_ENTRY_CATCH
}

int pic_adj_schedule(pic_adj* a, int32_t* absorb, size_t n) {
  PIC_ENTRY_TRY
  if (!a || !absorb || n != (size_t)a->np || !a->recorded) return PIC_EINVAL;
  CKA(cudaStreamSynchronize(a->st));
  CKA(cudaMemcpy(absorb, a->absorb, sizeof(int32_t) * n, cudaMemcpyDeviceToHost));
  return PIC_OK;
  PIC_ENTRY_CATCH
}

int pic_adj_tape(pic_adj* a, int32_t n, int32_t* cell, float* frac, float* vx, float* vy, float* vz, double* E,
                 size_t np, size_t nnodes) {
  PIC_ENTRY_TRY
  if (!a || !a->recorded || n < 0 || n > a->T || np != (size_t)a->np || nnodes != (size_t)a->N + 1) return PIC_EINVAL;
  pic_config c;
  const Phys ph = physics(a, a->rec_VL, a->rec_Te, &c);
  // the state after n steps: recomputed from its segment's checkpoint with the recorded fields (the
  // same kernel and inputs as the recording forward, so the same bits)
  const int seg = std::min(n / a->K, a->nseg - 1);
  const int n0 = seg * a->K;
  int rc = copy_state(a, a->tape[0], a->ckpt[seg]);
  if (rc != PIC_OK) return rc;
  AdjStep S = step_params(a, ph, c);
  S.mode = 2;
  for (int k = n0; k < n; ++k) {
    S.src = a->tape[k - n0];
    S.dst = a->tape[k + 1 - n0];
    S.E = a->Etape + (size_t)k * nnodes;
    S.step = k;
    CKA(launch_adj_push(S, a->max_grid, a->st));
  }
  CKA(cudaStreamSynchronize(a->st));
  const AdjState& t = a->tape[n - n0];
  if (cell) CKA(cudaMemcpy(cell, t.cell, 4 * np, cudaMemcpyDeviceToHost));
  if (frac) CKA(cudaMemcpy(frac, t.frac, 4 * np, cudaMemcpyDeviceToHost));
  if (vx) CKA(cudaMemcpy(vx, t.vx, 4 * np, cudaMemcpyDeviceToHost));
  if (vy) CKA(cudaMemcpy(vy, t.vy, 4 * np, cudaMemcpyDeviceToHost));
  if (vz) CKA(cudaMemcpy(vz, t.vz, 4 * np, cudaMemcpyDeviceToHost));
  if (E) CKA(cudaMemcpy(E, a->Etape + (size_t)n * nnodes, sizeof(double) * nnodes, cudaMemcpyDeviceToHost));
  return PIC_OK;
  PIC_ENTRY_CATCH
}

int pic_adj_times(pic_adj* a, double* forward_ms, double* gradient_ms) {
  PIC_ENTRY_TRY
  if (!a) return PIC_EINVAL;
  if (forward_ms) *forward_ms = a->ms_fwd;
  if (gradient_ms) *gradient_ms = a->ms_rev;
  return PIC_OK;
  PIC_ENTRY_CATCH
}

void pic_adj_free(pic_adj* a) {
  if (!a) return;
  cudaStreamSynchronize(a->st);
  if (a->owns_ws && a->ws) cudaFree(a->ws);
  delete a;
}

}  // extern "C"
