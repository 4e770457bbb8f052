// api.cu -- the C ABI of include/pic.h: configuration checks, device workspace layout, the
// per-step launch sequence, snapshot/restore (checkpoint/restart semantics of the paper's
// Sec. 4.1), diagnostics and kernel timing.  All device work is in the k_*.cu kernels.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <numeric>
#include <thread>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "api_internal.h"

namespace picx {

const char* const kKindNames[PIC_KERNEL_KINDS] = {"step", "source", "field", "sort", "load", "diag", "plan",
                                                   "step_scatter", "neutral", "neutral_compact"};


// ---------------------------------------------------------------------------------------------
bool valid(const pic_config* c) {
  if (!c || c->abi_version != PIC_ABI_VERSION) return false;
  if (c->precision > PIC_FP64_PLAIN) return false;
  if (c->ncells < 2 || c->ncells > PIC_MAX_CELLS_FP32) return false;
  if (!(c->L > 0) || !(c->dt > 0) || !std::isfinite(c->L) || !std::isfinite(c->dt)) return false;
  for (int s = 0; s < 2; ++s) {
    if (c->ppc[s] < 1 || !(c->mass[s] > 0) || !(c->T[s] >= 0) || c->charge[s] == 0) return false;
  }
  if (c->sort_interval < 1 || c->field_mode > PIC_FIELD_ZERO) return false;
  if (c->load_profile < 0 || c->load_profile > PIC_LOAD_QUIET_SINE) return false;
  if (c->load_profile == PIC_LOAD_EXP && !(c->profile_scale > 0)) return false;
  if (c->source_mode < 0 || c->source_mode > PIC_SOURCE_PAIRS) return false;
  if (c->source_mode == PIC_SOURCE_PAIRS && !(c->source_x1 > 0 && c->source_x1 <= c->ncells)) return false;
  if (!(c->n_gas >= 0) || !(c->Tg >= 0) || !(c->m_gas > 0)) return false;
  if (!(c->capacity_factor >= 1.0) || !(c->capacity_factor <= 64.0)) return false;
  if ((c->coll_mask & PIC_COLL_EX) && !(c->E_ex > 0)) return false;
  if ((c->coll_mask & PIC_COLL_IZ) && !(c->E_iz > 0)) return false;
  const double n = (double)c->ppc[0] * c->ncells * c->capacity_factor;
  const double m = (double)c->ppc[1] * c->ncells * c->capacity_factor;
  if (n > 2.0e9 || m > 2.0e9) return false;  // u32 cell cursors
  // sheath physics: FP32 path with the integer-exact field solve only
  if (c->reserved != 0u || c->neutrals > 1u || c->smooth_passes < 0 || c->smooth_passes > PIC_MAX_SMOOTH)
    return false;
  if ((c->neutrals || c->smooth_passes) && (c->precision != PIC_FP32 || !exact_possible(*c))) return false;
  if (c->neutrals) {
    if (!(c->recycle >= 0.0 && c->recycle <= 1.0) || !(c->T_rec >= 0.0) || !(c->K_iz >= 0.0) ||
        !(c->T_sec >= 0.0) || c->neutral_ppc < 0 || !(c->neutral_capacity >= 1.0) || !(c->neutral_capacity <= 64.0))
      return false;
    if ((double)std::max(c->neutral_ppc, c->ppc[1]) * c->ncells * c->neutral_capacity > 2.0e9) return false;
  } else if (c->neutral_ppc != 0) {
    return false;
  }
  return true;
}

unsigned long long capacity(const pic_config* c, int s) {
  double n = std::ceil((double)c->ppc[s] * (double)c->ncells * c->capacity_factor);
  unsigned long long v = (unsigned long long)n + 4ull;
  return (v + 1023ull) & ~1023ull;
}

unsigned long long neutral_capacity(const pic_config* c) {
  if (!c->neutrals) return 0ull;
  const double n = std::ceil((double)std::max(c->neutral_ppc, c->ppc[1]) * (double)c->ncells * c->neutral_capacity);
  const unsigned long long v = (unsigned long long)n + 4ull;
  return (v + 1023ull) & ~1023ull;
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

void layout(pic_handle* h, char* base, size_t* total) {
  Carve cv{base};
  const int N = h->N;
  h->ctl = cv.take<Ctl>(1);
  if (!h->plain) {
    for (int b = 0; b < 2; ++b)
      for (int s = 0; s < 2; ++s) {
        Species32& a = h->a32[b][s];
        a.cell = cv.take<int>(h->cap[s]);
        a.frac = cv.take<float>(h->cap[s]);
        a.vx = cv.take<float>(h->cap[s]);
        a.vy = cv.take<float>(h->cap[s]);
        a.vz = cv.take<float>(h->cap[s]);
        a.id = cv.take<unsigned long long>(h->cap[s]);
      }
    h->stage = reinterpret_cast<char*>(h->a32[1][0].cell);
    h->stage_bytes = h->stage ? (size_t)(reinterpret_cast<char*>(h->a32[1][1].id + h->cap[1]) - h->stage) : 0;
    for (int s = 0; s < 2; ++s) {
      h->cnt[s] = cv.take<unsigned int>(N);
      h->S[s] = cv.take<unsigned long long>(N);
      h->cursor[s] = cv.take<unsigned int>(N);
    }
    h->E2 = cv.take<float2>(N);
    h->fgrid = cv.take<FieldGrid>(1);
    if (h->cap_nt) {
      for (int b = 0; b < 2; ++b) {
        Species32& a = h->nt[b];
        a.cell = cv.take<int>(h->cap_nt);
        a.frac = cv.take<float>(h->cap_nt);
        a.vx = cv.take<float>(h->cap_nt);
        a.vy = cv.take<float>(h->cap_nt);
        a.vz = cv.take<float>(h->cap_nt);
        a.id = cv.take<unsigned long long>(h->cap_nt);
      }
      h->NE2 = cv.take<float2>(N);
      h->wlog = cv.take<unsigned int>(h->cap[1]);
    }
  } else {
    for (int s = 0; s < 2; ++s) {
      Species64& a = h->a64[s];
      a.x = cv.take<double>(h->cap[s]);
      a.vx = cv.take<double>(h->cap[s]);
      a.vy = cv.take<double>(h->cap[s]);
      a.vz = cv.take<double>(h->cap[s]);
      a.id = cv.take<unsigned long long>(h->cap[s]);
      a.nk = cv.take<unsigned>(h->cap[s]);
    }
    for (int s = 0; s < 2; ++s) h->acc[s] = cv.take<double>(N + 1);
  }
  for (int s = 0; s < 2; ++s) h->R[s] = cv.take<long long>(N + 1);
  h->rho = cv.take<double>(N + 1);
  h->phi = cv.take<double>(N + 1);
  h->E = cv.take<double>(N + 1);
  *total = cv.off + 256;
}

// Physics constants (host, FP64), rounded once to FP32 for the FP32 path.  The null-collision
// bound nu_max = n_g * sum(sigma_max) * v_cap, v_cap = sqrt(2 (E_cap + |V_L - V_R|) / m), is rounded to
// FP32 first and P_null = 1 - exp(-nu_max dt) is computed from that FP32 value.
void derive(pic_handle* h) {
  const pic_config& c = h->cfg;
  Phys& p = h->ph;
  std::memset(&p, 0, sizeof(p));
  const double dx = c.L / c.ncells;
  const double th = c.B_angle_deg * 3.14159265358979323846 / 180.0;
  const double Bv[3] = {c.B * std::cos(th), c.B * std::sin(th), 0.0};
  const double Ecap = c.E_cap + std::fabs(c.V_left - c.V_right);
  double smax[2];
  smax[0] = ((c.coll_mask & PIC_COLL_EL) ? c.sigma_el : 0.0) + ((c.coll_mask & PIC_COLL_EX) ? c.sigma_ex : 0.0) +
            ((c.coll_mask & PIC_COLL_IZ) ? c.sigma_iz : 0.0);
  smax[1] = (c.coll_mask & PIC_COLL_CX) ? c.sigma_cx : 0.0;
  for (int s = 0; s < 2; ++s) {
    SpConst& k = p.sp[s];
    const double h2 = 0.5 * (c.charge[s] / c.mass[s]) * c.dt;
    double t[3], tt = 0.0;
    for (int i = 0; i < 3; ++i) {
      t[i] = h2 * Bv[i];
      tt += t[i] * t[i];
    }
    for (int i = 0; i < 3; ++i) {
      k.t_d[i] = t[i];
      k.s_d[i] = 2.0 * t[i] / (1.0 + tt);
      k.t[i] = (float)k.t_d[i];
      k.s[i] = (float)k.s_d[i];
    }
    k.qmdt2_d = h2;
    k.qmdt2 = (float)h2;
    k.mass_d = c.mass[s];
    k.mass = (float)c.mass[s];
    k.vt_d = std::sqrt(c.T[s] / c.mass[s]);
    k.vt = (float)k.vt_d;
    k.w = (float)(dx / c.ppc[s]);
    k.qsign = c.charge[s] > 0 ? 1 : -1;
    const double vcap = std::sqrt(2.0 * Ecap / c.mass[s]);
    k.nu_max = (float)(c.n_gas * smax[s] * vcap);
    k.p_null = (float)(1.0 - std::exp(-(double)k.nu_max * c.dt));
    k.p_null_u24 = (unsigned)std::ceil((double)k.p_null * 16777216.0);
    k.lnq_d = std::log1p(-(double)k.p_null);  // the countdown's geometric parameter
    k.lnq = (float)k.lnq_d;
  }
  p.dtdx_d = c.dt / dx;
  p.dtdx = (float)p.dtdx_d;
  p.ngs_el_d = c.n_gas * c.sigma_el;
  p.ngs_ex_d = c.n_gas * c.sigma_ex;
  p.ngs_iz_d = c.n_gas * c.sigma_iz;
  p.ngs_cx_d = c.n_gas * c.sigma_cx;
  p.ngs_el = (float)p.ngs_el_d;
  p.ngs_ex = (float)p.ngs_ex_d;
  p.ngs_iz = (float)p.ngs_iz_d;
  p.ngs_cx = (float)p.ngs_cx_d;
  p.E_ex_d = c.E_ex;
  p.E_iz_d = c.E_iz;
  p.E_ex = (float)c.E_ex;
  p.E_iz = (float)c.E_iz;
  p.inv_E_ex = c.E_ex > 0 ? (float)(1.0 / c.E_ex) : 0.f;
  p.inv_E_iz = c.E_iz > 0 ? (float)(1.0 / c.E_iz) : 0.f;
  p.two_m_over_M_d = 2.0 * c.mass[0] / c.m_gas;
  p.two_m_over_M = (float)p.two_m_over_M_d;
  p.vt_gas_d = std::sqrt(c.Tg / c.mass[1]);
  p.vt_gas = (float)p.vt_gas_d;
  p.E_ext_d = c.E_ext;
  p.E_ext = (float)c.E_ext;
  p.src_x1_d = c.source_x1;
  p.src_x1 = (float)c.source_x1;
  p.coll_mask = c.coll_mask;
  p.field_mode = c.field_mode;
  p.push_mask = 3u & ~c.frozen_mask;
  p.has_B = c.B != 0.0 ? 1u : 0u;
  p.mcc_mask = 0u;
  for (int s = 0; s < 2; ++s) {  // species that take the null-collision test (and carry a countdown)
    const bool on = s == 0 ? (c.coll_mask & (PIC_COLL_EL | PIC_COLL_EX | PIC_COLL_IZ)) != 0u
                           : (c.coll_mask & PIC_COLL_CX) != 0u;
    if (on && ((p.push_mask >> s) & 1u) && p.sp[s].p_null > 0.f) p.mcc_mask |= 1u << s;
  }
  p.N = c.ncells;
  p.seed = c.seed;
}

// ---------------------------------------------------------------------------------------------
void prof_begin(pic_handle* h, int kind, EvPair* e) {
  nvtxRangePushA(kKindNames[kind]);  // a named range per launch for timeline tools (no tool: a no-op)
  e->kind = kind;
  e->a = e->b = nullptr;
  if (!h->prof) return;
  for (cudaEvent_t* x : {&e->a, &e->b}) {
    if (!h->ev_free.empty()) {
      *x = h->ev_free.back();
      h->ev_free.pop_back();
    } else if (cudaEventCreate(x) != cudaSuccess) {
      *x = nullptr;
    }
  }
  if (!e->a || !e->b) {  // no event: this launch goes untimed
    if (e->a) h->ev_free.push_back(e->a);
    if (e->b) h->ev_free.push_back(e->b);
    e->a = e->b = nullptr;
    return;
  }
  cudaEventRecord(e->a, h->st);
}

void prof_end(pic_handle* h, EvPair* e) {
  nvtxRangePop();
  if (!h->prof || !e->a) return;
  cudaEventRecord(e->b, h->st);
  h->ev.push_back(*e);
}

void prof_harvest(pic_handle* h) {
  for (EvPair& e : h->ev) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, e.a, e.b) == cudaSuccess) {
      h->ms[e.kind] += ms;
      h->launches[e.kind] += 1;
    }
    h->ev_free.push_back(e.a);
    h->ev_free.push_back(e.b);
  }
  h->ev.clear();
}

// The tensor maps of the particle step's stage loads (StepMaps), made once per handle: per buffer
// and species, the five 4-byte arrays as a 2-D tensor of 32-bit elements, cap[s] wide and 5 rows,
// the rows as far apart as the workspace layout places the arrays (cap[s] elements in a single
// run; the whole batch's capacity in a run of an ensemble), read in boxes of 128 x 5.  The encoder
// is the driver's cuTensorMapEncodeTiled, reached through the runtime.  Until the maps exist
// (maps_ok) no particle step is launched for the handle.
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_tiled() {
  static EncodeTiledFn fn = [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess) {
      cudaGetLastError();
      return (EncodeTiledFn) nullptr;
    }
    return reinterpret_cast<EncodeTiledFn>(p);
  }();
  return fn;
}

int encode_step_maps(const Species32* a, const unsigned long long* cap, StepMaps* out) {
  const EncodeTiledFn enc = encode_tiled();
  if (!enc) return PIC_ECUDA;
  for (int s = 0; s < 2; ++s) {
    const char* const rows[5] = {reinterpret_cast<const char*>(a[s].cell), reinterpret_cast<const char*>(a[s].frac),
                                 reinterpret_cast<const char*>(a[s].vx), reinterpret_cast<const char*>(a[s].vy),
                                 reinterpret_cast<const char*>(a[s].vz)};
    const long long pitch = rows[1] - rows[0];
    bool ok = pitch >= (long long)(cap[s] * 4) && pitch % 16 == 0 && (reinterpret_cast<uintptr_t>(rows[0]) & 15u) == 0;
    for (int r = 2; r < 5; ++r) ok = ok && rows[r] - rows[r - 1] == pitch;
    if (!ok) return PIC_ECUDA;  // not a layout the maps can describe
    const cuuint64_t dims[2] = {cap[s], 5};
    const cuuint64_t strides[1] = {(cuuint64_t)pitch};
    const cuuint32_t box[2] = {32 * PIC_PPT, 5};
    const cuuint32_t estr[2] = {1, 1};
    if (enc(&out->tmap[s], CU_TENSOR_MAP_DATA_TYPE_UINT32, 2, a[s].cell, dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return PIC_ECUDA;
  }
  return PIC_OK;
}

int make_step_maps(pic_handle* h) {
  h->maps_ok = false;
  for (int b = 0; b < 2; ++b) {
    const int rc = encode_step_maps(h->a32[b], h->cap, &h->maps[b]);
    if (rc != PIC_OK) return rc;
  }
  h->maps_ok = true;
  return PIC_OK;
}

StepParams32 params32(pic_handle* h) {
  StepParams32 P;
  for (int s = 0; s < 2; ++s) {
    P.sp[s] = h->a32[h->cur][s];
    P.cap[s] = h->cap[s];
    P.cnt[s] = h->cnt[s];
    P.S[s] = h->S[s];
  }
  P.E2 = h->E2;
  P.ctl = h->ctl;
  P.ph = h->ph;
  P.step = h->step;
  P.sum_ke = 0u;
  P.scatter = 0u;
  for (int s = 0; s < 2; ++s) {
    P.src[s] = P.sp[s];
    P.cursor[s] = h->cursor[s];
  }
  P.wlog = (h->cap_nt && h->cfg.recycle > 0.0) ? h->wlog : nullptr;
  return P;
}

// The neutral step of a particle step with parameters P (its charged buffers and counters).
NeutralParams neutral_params(pic_handle* h, const StepParams32& P) {
  NeutralParams Q;
  std::memset(&Q, 0, sizeof(Q));
  const pic_config& c = h->cfg;
  Q.P = P;
  Q.src = h->nt[h->nt_buf];
  Q.dst = h->nt[1 - h->nt_buf];
  Q.cap = h->cap_nt;
  Q.ion_id = P.src[1].id;
  Q.NE2 = h->NE2;
  Q.Kdt = (float)(c.K_iz * c.dt);
  Q.vt_rec = (float)std::sqrt(c.T_rec / c.mass[1]);
  Q.vt_sec = (float)std::sqrt(c.T_sec / c.mass[0]);
  Q.mass = (float)c.mass[1];
  Q.recycle_u24 = (unsigned)std::ceil(c.recycle * 16777216.0);
  Q.ionize = c.K_iz > 0.0 ? 1 : 0;
  return Q;
}

StepParams64 params64(pic_handle* h) {
  StepParams64 P;
  for (int s = 0; s < 2; ++s) {
    P.sp[s] = h->a64[s];
    P.cap[s] = h->cap[s];
    P.acc[s] = h->acc[s];
  }
  P.E = h->E;
  P.ctl = h->ctl;
  P.ph = h->ph;
  P.step = h->step;
  return P;
}

// Integer-exact field (k_field_exact) when both charges are small integers: the net deposit
// r = m_0 R_0 + m_1 R_1 with m_s = q_s ppc_{1-s} / g (g = gcd of the ppc) is an exact integer and
// f = kappa r with kappa = dx^2 2^-32 g / (ppc_0 ppc_1).
bool exact_possible(const pic_config& c) {
  const long long g = std::gcd((long long)c.ppc[0], (long long)c.ppc[1]);
  for (int s = 0; s < 2; ++s) {
    const double q = c.charge[s];
    if (q != std::floor(q) || std::fabs(q) > 64.0) return false;
    if ((long long)c.ppc[1 - s] / g > 1024) return false;
  }
  return true;
}

void exact_coefficients(pic_handle* h, PoissonParams* F) {
  const pic_config& c = h->cfg;
  F->exact = 0;
  if (h->plain || !exact_possible(c)) return;
  long long g = std::gcd((long long)c.ppc[0], (long long)c.ppc[1]);
  for (int s = 0; s < 2; ++s) {
    const double q = c.charge[s];
    if (q != std::floor(q) || std::fabs(q) > 64.0) return;
    const long long other = (long long)c.ppc[1 - s] / g;
    if (other > 1024) return;
    F->m[s] = (long long)q * other;
  }
  const int N = c.ncells;
  const double dx = c.L / N;
  const double kappa = dx * dx * 2.3283064365386963e-10 * (double)g / ((double)c.ppc[0] * (double)c.ppc[1]);
  // smoothing leaves the net charge in units of 2^-(2 passes + 1) of the deposit unit
  const double unit = c.smooth_passes > 0 ? std::ldexp(1.0, -(2 * c.smooth_passes + 1)) : 1.0;
  F->e_in = unit * kappa / (2.0 * N * dx);
  F->e_wall = unit * kappa / ((double)N * dx);
  F->e_bias = (c.V_left - c.V_right) / ((double)N * dx);
  F->exact = 1;
}

PoissonParams field_params(pic_handle* h, bool keep_counts, bool count_step) {
  PoissonParams F;
  std::memset(&F, 0, sizeof(F));
  const double dx = h->cfg.L / h->cfg.ncells;
  for (int s = 0; s < 2; ++s) {
    F.cnt[s] = h->cnt[s];
    F.S[s] = h->S[s];
    F.acc[s] = h->acc[s];
    F.qw[s] = h->cfg.charge[s] * (dx / h->cfg.ppc[s]);
    F.R[s] = h->R[s];
    F.cap[s] = h->cap[s];
    if (!h->plain) F.pad32[s] = h->a32[h->cur][s];
    F.pad64[s] = h->a64[s];
  }
  F.mode = h->plain ? 1 : 0;
  F.inv_dx = 1.0 / dx;
  exact_coefficients(h, &F);
  F.keep_counts = keep_counts ? 1 : 0;
  F.count_step = count_step ? 1 : 0;
  F.N = h->N;
  F.dx = dx;
  F.V_L = h->cfg.V_left;
  F.V_R = h->cfg.V_right;
  F.rho = h->rho;
  F.phi = h->phi;
  F.E = h->E;
  F.E2 = h->E2;
  F.ctl = h->ctl;
  F.plain = h->plain ? 1 : 0;
  F.smooth = h->cfg.smooth_passes;
  F.NE2 = h->NE2;
  F.ne_scale = (dx / h->cfg.ppc[0]) * 2.3283064365386963e-10 / dx;
  F.nt_cap = h->cap_nt;
  F.grid = h->field_ctas > 0 ? h->fgrid : nullptr;
  F.grid_ctas = h->field_ctas;
  return F;
}

#define CK(x)                                \
  do {                                       \
    cudaError_t e__ = (x);                   \
    if (e__ != cudaSuccess) return PIC_ECUDA; \
  } while (0)

// Deposit of the current particles without moving them, field solve, and (FP32) the sort.
int refresh_field(pic_handle* h) {
  EvPair e;
  Phys saved = h->ph;
  h->ph.push_mask = 0u;
  h->ph.coll_mask = 0u;
  prof_begin(h, K_STEP, &e);
  StepParams32 P32 = params32(h);
  P32.sum_ke = 1u;
  cudaError_t err = h->plain ? launch_step64(params64(h), h->grid_step, h->st)
                             : (h->maps_ok ? launch_step32(P32, h->maps[h->cur], h->grid_step, h->st)
                                           : cudaErrorInvalidValue);
  prof_end(h, &e);
  h->ph = saved;
  h->ke_valid = !h->plain;
  h->pending_scatter = false;  // the full sort below replaces any pending one
  CK(err);
  prof_begin(h, K_FIELD, &e);
  CK(launch_field(field_params(h, !h->plain, false), h->st));
  prof_end(h, &e);
  if (!h->plain) {
    prof_begin(h, K_SORT, &e);
    Species32 src[2] = {h->a32[h->cur][0], h->a32[h->cur][1]};
    Species32 dst[2] = {h->a32[1 - h->cur][0], h->a32[1 - h->cur][1]};
    CK(launch_sort32(src, dst, h->cnt, h->cursor, h->cap, h->ctl, h->N, h->grid_sort, h->st));
    prof_end(h, &e);
    h->cur = 1 - h->cur;
  }
  return PIC_OK;
}

// rho and phi of the current deposit, from the stored node deposits (FP64 Green's function);
// the node field the particles use is left as the step computed it.
int field_diagnostics(pic_handle* h) {
  PoissonParams F = field_params(h, true, false);
  F.mode = 3;
  F.ctl = nullptr;
  F.E = nullptr;
  F.E2 = nullptr;
  if (h->plain) return PIC_OK;  // the plain path's solve already produced rho and phi
  CK(launch_field(F, h->st));
  return PIC_OK;
}

int status_of(unsigned int err) {
  if (err & ERR_OVERFLOW) return PIC_EOVERFLOW;
  if (err & ERR_TIMEOUT) return PIC_ETIMEOUT;
  if (err & ERR_DEVICE) return PIC_EDEVICE;
  return PIC_OK;
}

int check_errors(pic_handle* h) {
  CK(cudaStreamSynchronize(h->st));
  unsigned int err = 0;
  CK(cudaMemcpy(&err, &h->ctl->error, sizeof(err), cudaMemcpyDeviceToHost));
  return status_of(err);
}

int load_initial(pic_handle* h) {
  const pic_config& c = h->cfg;
  int rc = PIC_OK;
  h->cur = 0;
  h->step = 0;
  unsigned long long n[2];
  for (int s = 0; s < 2; ++s) n[s] = (unsigned long long)c.ppc[s] * (unsigned long long)c.ncells;
  {
    EvPair e;
    prof_begin(h, K_LOAD, &e);
    cudaError_t err = h->plain ? launch_load64(params64(h), n, c.load_profile, c.ppc[0], c.ppc[1],
                                               c.profile_scale, c.profile_mode, h->st)
                               : launch_load32(params32(h), n, c.load_profile, c.ppc[0], c.ppc[1],
                                               c.profile_scale, c.profile_mode, h->st);
    prof_end(h, &e);
    if (err != cudaSuccess) rc = PIC_ECUDA;
  }
  if (rc == PIC_OK) {
    // extents, padding slots, live counts
    Ctl c0;
    std::memset(&c0, 0, sizeof(c0));
    for (int s = 0; s < 2; ++s) {
      c0.n_cur[s] = round_up4(n[s]);
      c0.n_live[s] = n[s];
      const unsigned long long pad = c0.n_cur[s] - n[s];
      if (pad) {
        if (!h->plain) {
          int dead[4] = {PIC_DEAD_CELL, PIC_DEAD_CELL, PIC_DEAD_CELL, PIC_DEAD_CELL};
          if (cudaMemcpyAsync(h->a32[0][s].cell + n[s], dead, pad * 4, cudaMemcpyHostToDevice, h->st) != cudaSuccess)
            rc = PIC_ECUDA;
        } else {
          double dead[4] = {-1.0, -1.0, -1.0, -1.0};
          if (cudaMemcpyAsync(h->a64[s].x + n[s], dead, pad * 8, cudaMemcpyHostToDevice, h->st) != cudaSuccess)
            rc = PIC_ECUDA;
        }
      }
    }
    if (rc == PIC_OK && h->cap_nt) {  // initial neutrals into buffer 0
      h->nt_buf = 0;
      const unsigned long long nn = (unsigned long long)c.neutral_ppc * (unsigned long long)c.ncells;
      if (round_up4(nn) > h->cap_nt) {
        rc = PIC_EOVERFLOW;
      } else {
        EvPair e;
        prof_begin(h, K_LOAD, &e);
        if (launch_nload32(h->nt[0], nn, c.neutral_ppc, c.ncells, c.seed, std::sqrt(c.T_rec / c.mass[1]), h->st) !=
            cudaSuccess)
          rc = PIC_ECUDA;
        prof_end(h, &e);
        const int dead[4] = {PIC_DEAD_CELL, PIC_DEAD_CELL, PIC_DEAD_CELL, PIC_DEAD_CELL};
        if (rc == PIC_OK && round_up4(nn) > nn &&
            cudaMemcpyAsync(h->nt[0].cell + nn, dead, 4 * (round_up4(nn) - nn), cudaMemcpyHostToDevice, h->st) !=
                cudaSuccess)
          rc = PIC_ECUDA;
        c0.nt_cur = round_up4(nn);
        c0.nt_live = nn;
      }
    }
    if (rc == PIC_OK && cudaMemcpyAsync(h->ctl, &c0, sizeof(c0), cudaMemcpyHostToDevice, h->st) != cudaSuccess)
      rc = PIC_ECUDA;
    if (rc == PIC_OK) rc = cudaStreamSynchronize(h->st) == cudaSuccess ? PIC_OK : PIC_ECUDA;  // c0 is on the stack
    if (rc == PIC_OK) rc = refresh_field(h);
    if (rc == PIC_OK) rc = check_errors(h);
  }
  return rc;
}

// ---------------------------------------------------------------------------------------------
// Snapshot format helpers (CRC-32 IEEE 802.3 reflected; FNV-1a 64 of the canonical config).
// CRC-32 (IEEE 802.3, reflected polynomial 0xEDB88320, as zlib), slice-by-8 tables.
struct CrcTables {
  uint32_t t[8][256];
  CrcTables() {
    for (uint32_t i = 0; i < 256; ++i) {
      uint32_t c = i;
      for (int k = 0; k < 8; ++k) c = (c & 1u) ? 0xEDB88320u ^ (c >> 1) : (c >> 1);
      t[0][i] = c;
    }
    for (uint32_t i = 0; i < 256; ++i)
      for (int k = 1; k < 8; ++k) t[k][i] = t[0][t[k - 1][i] & 0xFFu] ^ (t[k - 1][i] >> 8);
  }
};
const CrcTables& crc_tables() {
  static const CrcTables T;
  return T;
}

// One slice-by-8 step of the raw (uncomplemented) CRC register.
inline uint32_t crc_step8(const CrcTables& T, uint32_t c, const unsigned char* p) {
  uint32_t lo, hi;
  std::memcpy(&lo, p, 4);
  std::memcpy(&hi, p + 4, 4);
  lo ^= c;
  return T.t[7][lo & 0xFF] ^ T.t[6][(lo >> 8) & 0xFF] ^ T.t[5][(lo >> 16) & 0xFF] ^ T.t[4][lo >> 24] ^
         T.t[3][hi & 0xFF] ^ T.t[2][(hi >> 8) & 0xFF] ^ T.t[1][(hi >> 16) & 0xFF] ^ T.t[0][hi >> 24];
}

uint32_t crc_raw(const CrcTables& T, uint32_t c, const unsigned char* p, size_t n) {
  while (n >= 8) {
    c = crc_step8(T, c, p);
    p += 8;
    n -= 8;
  }
  while (n--) c = T.t[0][(c ^ *p++) & 0xFFu] ^ (c >> 8);
  return c;
}

uint32_t crc32_join(uint32_t crc_a, uint32_t crc_b, size_t len_b);

// The CRC of one thread's part.  Each step of a single register depends on the one before, so the
// part is split into four quarters whose registers advance together (four independent chains of
// table loads) and the four CRCs are joined: 2.4x the single-chain rate on one core.
uint32_t crc32_serial(const unsigned char* p, size_t n) {
  const CrcTables& T = crc_tables();
  const size_t q = (n / 4) & ~size_t(7);
  if (q < 4096) return crc_raw(T, 0xFFFFFFFFu, p, n) ^ 0xFFFFFFFFu;
  const unsigned char *p0 = p, *p1 = p + q, *p2 = p + 2 * q, *p3 = p + 3 * q;
  uint32_t c0 = 0xFFFFFFFFu, c1 = c0, c2 = c0, c3 = c0;
  for (size_t i = 0; i < q; i += 8) {
    c0 = crc_step8(T, c0, p0 + i);
    c1 = crc_step8(T, c1, p1 + i);
    c2 = crc_step8(T, c2, p2 + i);
    c3 = crc_step8(T, c3, p3 + i);
  }
  c3 = crc_raw(T, c3, p3 + q, n - 4 * q);
  uint32_t c = crc32_join(c0 ^ 0xFFFFFFFFu, c1 ^ 0xFFFFFFFFu, q);
  c = crc32_join(c, c2 ^ 0xFFFFFFFFu, q);
  return crc32_join(c, c3 ^ 0xFFFFFFFFu, n - 3 * q);
}

// GF(2) operator on the CRC register, column i = image of bit i.
struct Gf2 {
  uint32_t m[32];
};
uint32_t gf2_apply(const Gf2& a, uint32_t v) {
  uint32_t r = 0;
  for (int i = 0; v; ++i, v >>= 1)
    if (v & 1u) r ^= a.m[i];
  return r;
}
Gf2 gf2_square(const Gf2& a) {
  Gf2 r;
  for (int i = 0; i < 32; ++i) r.m[i] = gf2_apply(a, a.m[i]);
  return r;
}
// crc(A || B) = crc(B) xor Z^{|B|}(crc(A)), Z = the register update of one zero byte (the init and
// final complements cancel), so chunks can be checksummed independently and joined.
uint32_t crc32_join(uint32_t crc_a, uint32_t crc_b, size_t len_b) {
  Gf2 op;
  op.m[0] = 0xEDB88320u;  // one zero bit: r -> (r >> 1) ^ (r & 1 ? P : 0)
  for (int i = 1; i < 32; ++i) op.m[i] = 1u << (i - 1);
  op = gf2_square(gf2_square(gf2_square(op)));  // one zero byte
  while (len_b) {
    if (len_b & 1u) crc_a = gf2_apply(op, crc_a);
    op = gf2_square(op);
    len_b >>= 1;
  }
  return crc_a ^ crc_b;
}

// Host threads for the large linear passes over a blob (checksum, range checks).
int host_threads(size_t bytes) {
  const unsigned hw = std::thread::hardware_concurrency();
  const size_t by_size = bytes / (32u << 20) + 1;  // at least 32 MB per thread
  return (int)std::max<size_t>(1, std::min<size_t>({by_size, (size_t)(hw ? hw : 1), (size_t)64}));
}

uint32_t crc32_ieee(const unsigned char* p, size_t n) {
  const int T = host_threads(n);
  if (T == 1) return crc32_serial(p, n);
  std::vector<uint32_t> part(T);
  std::vector<size_t> len(T);
  std::vector<std::thread> th;
  const size_t chunk = (n + T - 1) / T;
  for (int k = 0; k < T; ++k) {
    const size_t a = std::min(n, (size_t)k * chunk), b = std::min(n, a + chunk);
    len[k] = b - a;
    th.emplace_back([&, k, a]() { part[k] = crc32_serial(p + a, len[k]); });
  }
  for (auto& t : th) t.join();
  uint32_t c = part[0];
  for (int k = 1; k < T; ++k) c = crc32_join(c, part[k], len[k]);
  return c;
}

struct Fnv {
  uint64_t h = 0xcbf29ce484222325ull;
  void add(const void* p, size_t n) {
    const unsigned char* b = static_cast<const unsigned char*>(p);
    for (size_t i = 0; i < n; ++i) {
      h ^= b[i];
      h *= 0x100000001b3ull;
    }
  }
};

// Canonical physics fields (precision, sort interval and capacities excluded): int32 ncells,
// ppc[2], load_profile, profile_mode, source_mode; uint32 coll_mask, field_mode, frozen_mask;
// f64 L, dt, mass[2], charge[2], T[2], Tg, m_gas, B, B_angle_deg, V_left, V_right, n_gas,
// sigma_el, sigma_ex, E_ex, sigma_iz, E_iz, sigma_cx, E_cap, E_ext, profile_scale, source_x1;
// u64 seed; then, when smoothing or neutrals are on, int32 smooth_passes, neutrals, neutral_ppc;
// f64 recycle, T_rec, K_iz, T_sec; all little-endian.
uint64_t config_hash(const pic_config& c) {
  Fnv f;
  const int32_t iv[6] = {c.ncells, c.ppc[0], c.ppc[1], c.load_profile, c.profile_mode, c.source_mode};
  const uint32_t uv[3] = {c.coll_mask, c.field_mode, c.frozen_mask};
  const double dv[25] = {c.L,        c.dt,          c.mass[0], c.mass[1],  c.charge[0], c.charge[1], c.T[0],
                         c.T[1],     c.Tg,          c.m_gas,   c.B,        c.B_angle_deg, c.V_left,   c.V_right,
                         c.n_gas,    c.sigma_el,    c.sigma_ex, c.E_ex,    c.sigma_iz,  c.E_iz,      c.sigma_cx,
                         c.E_cap,    c.E_ext,       c.profile_scale,       c.source_x1};
  f.add(iv, sizeof(iv));
  f.add(uv, sizeof(uv));
  f.add(dv, sizeof(dv));
  f.add(&c.seed, sizeof(c.seed));
  if (c.smooth_passes || c.neutrals) {  // the sheath-physics fields, when any is in use
    const int32_t iv2[3] = {c.smooth_passes, (int32_t)c.neutrals, c.neutral_ppc};
    const double dv2[4] = {c.recycle, c.T_rec, c.K_iz, c.T_sec};
    f.add(iv2, sizeof(iv2));
    f.add(dv2, sizeof(dv2));
  }
  return f.h;
}

const size_t kHdr = 8 + 4 + 4 + 8 + 8 + 16 + 17 * 8 + 8 + 16;
const size_t kNtHdr = 8 + 6 * 8;  // version 2: u64 n_neutral, u64 recycled[2], lost[2], ionized, near

struct HostParticles {
  std::vector<int32_t> cell;
  std::vector<double> frac, vx, vy, vz;
  std::vector<uint64_t> id;
};

// fn(lo, hi) over [0, n) split into contiguous ranges, one per host thread (sized by the bytes
// the pass touches).
template <class F>
void host_parallel(size_t n, size_t bytes_per_item, F fn) {
  const int T = host_threads(n * bytes_per_item);
  if (T <= 1) {
    fn((size_t)0, n);
    return;
  }
  std::vector<std::thread> th;
  const size_t chunk = (n + T - 1) / T;
  for (int k = 0; k < T; ++k) {
    const size_t lo = std::min(n, (size_t)k * chunk), hi = std::min(n, lo + chunk);
    th.emplace_back([lo, hi, &fn]() { fn(lo, hi); });
  }
  for (auto& t : th) t.join();
}

struct IdIdx {
  uint64_t id, i;
};

// The live entries (cell != PIC_DEAD_CELL) of n as (id, index) pairs in ascending id order.  Ids
// are unique, so the order is unique: each host thread collects and sorts the pairs of its range,
// then neighbouring sorted runs are merged in parallel rounds.
std::vector<IdIdx> live_by_id(const int32_t* cell, const uint64_t* id, size_t n) {
  const int T = std::max(1, host_threads(12 * n));
  const size_t chunk = (n + T - 1) / T;
  std::vector<size_t> cnt(T + 1, 0);
  {
    std::vector<std::thread> th;
    for (int k = 0; k < T; ++k)
      th.emplace_back([&, k]() {
        const size_t lo = std::min(n, (size_t)k * chunk), hi = std::min(n, lo + chunk);
        size_t c = 0;
        for (size_t i = lo; i < hi; ++i) c += cell[i] != PIC_DEAD_CELL;
        cnt[k + 1] = c;
      });
    for (auto& t : th) t.join();
  }
  for (int k = 0; k < T; ++k) cnt[k + 1] += cnt[k];
  std::vector<IdIdx> a(cnt[T]), b;
  const auto by_id = [](const IdIdx& x, const IdIdx& y) { return x.id < y.id; };
  {
    std::vector<std::thread> th;
    for (int k = 0; k < T; ++k)
      th.emplace_back([&, k]() {
        const size_t lo = std::min(n, (size_t)k * chunk), hi = std::min(n, lo + chunk);
        size_t o = cnt[k];
        for (size_t i = lo; i < hi; ++i)
          if (cell[i] != PIC_DEAD_CELL) a[o++] = IdIdx{id[i], (uint64_t)i};
        std::sort(a.begin() + (std::ptrdiff_t)cnt[k], a.begin() + (std::ptrdiff_t)cnt[k + 1], by_id);
      });
    for (auto& t : th) t.join();
  }
  std::vector<size_t> run(cnt.begin(), cnt.end());  // run r is [run[r], run[r + 1])
  if (run.size() > 2) b.resize(a.size());
  while (run.size() > 2) {
    std::vector<size_t> next;
    std::vector<std::thread> th;
    for (size_t r = 0; r + 1 < run.size(); r += 2) {
      next.push_back(run[r]);
      const size_t lo = run[r], mid = run[r + 1], hi = r + 2 < run.size() ? run[r + 2] : run[r + 1];
      th.emplace_back([&, lo, mid, hi]() {
        std::merge(a.begin() + (std::ptrdiff_t)lo, a.begin() + (std::ptrdiff_t)mid, a.begin() + (std::ptrdiff_t)mid,
                   a.begin() + (std::ptrdiff_t)hi, b.begin() + (std::ptrdiff_t)lo, by_id);
      });
    }
    next.push_back(run.back());
    for (auto& t : th) t.join();
    a.swap(b);
    run.swap(next);
  }
  return a;
}

// Gathers the live particles of one species in ascending id order (cell, fraction, v as read).
template <class Frac, class Vel>
void gather_by_id(const std::vector<IdIdx>& live, const int32_t* cell, const Frac* frac, const Vel* vx,
                  const Vel* vy, const Vel* vz, HostParticles& o) {
  const size_t m = live.size();
  o.cell.resize(m);
  o.frac.resize(m);
  o.vx.resize(m);
  o.vy.resize(m);
  o.vz.resize(m);
  o.id.resize(m);
  host_parallel(m, 64, [&](size_t lo, size_t hi) {
    for (size_t k = lo; k < hi; ++k) {
      const size_t i = (size_t)live[k].i;
      o.cell[k] = cell[i];
      o.frac[k] = (double)frac[i];
      o.vx[k] = (double)vx[i];
      o.vy[k] = (double)vy[i];
      o.vz[k] = (double)vz[i];
      o.id[k] = live[k].id;
    }
  });
}

int fetch_particles(pic_handle* h, HostParticles out[2], Ctl* ctl) {
  CK(cudaStreamSynchronize(h->st));
  CK(cudaMemcpy(ctl, h->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost));
  for (int s = 0; s < 2; ++s) {
    const size_t n = (size_t)ctl->n_cur[s];
    std::vector<uint64_t> id(n);
    std::vector<int32_t> cell(n);
    if (!h->plain) {
      const Species32& a = h->a32[h->cur][s];
      std::vector<float> f(n), vx(n), vy(n), vz(n);
      CK(cudaMemcpy(cell.data(), a.cell, n * 4, cudaMemcpyDeviceToHost));
      CK(cudaMemcpy(f.data(), a.frac, n * 4, cudaMemcpyDeviceToHost));
      CK(cudaMemcpy(vx.data(), a.vx, n * 4, cudaMemcpyDeviceToHost));
      CK(cudaMemcpy(vy.data(), a.vy, n * 4, cudaMemcpyDeviceToHost));
      CK(cudaMemcpy(vz.data(), a.vz, n * 4, cudaMemcpyDeviceToHost));
      CK(cudaMemcpy(id.data(), a.id, n * 8, cudaMemcpyDeviceToHost));
      gather_by_id(live_by_id(cell.data(), id.data(), n), cell.data(), f.data(), vx.data(), vy.data(), vz.data(),
                   out[s]);
    } else {
      const Species64& a = h->a64[s];
      std::vector<double> x(n), vx(n), vy(n), vz(n);
      CK(cudaMemcpy(x.data(), a.x, n * 8, cudaMemcpyDeviceToHost));
      CK(cudaMemcpy(vx.data(), a.vx, n * 8, cudaMemcpyDeviceToHost));
      CK(cudaMemcpy(vy.data(), a.vy, n * 8, cudaMemcpyDeviceToHost));
      CK(cudaMemcpy(vz.data(), a.vz, n * 8, cudaMemcpyDeviceToHost));
      CK(cudaMemcpy(id.data(), a.id, n * 8, cudaMemcpyDeviceToHost));
      std::vector<unsigned> nk(n);
      CK(cudaMemcpy(nk.data(), a.nk, n * 4, cudaMemcpyDeviceToHost));
      // absolute x -> (cell word, fraction); absorbed particles carry x < 0
      host_parallel(n, 16, [&](size_t lo, size_t hi) {
        for (size_t i = lo; i < hi; ++i) {
          if (x[i] < 0.0) {
            cell[i] = PIC_DEAD_CELL;
            continue;
          }
          const double c = std::floor(x[i]);
          cell[i] = (int32_t)((uint32_t)c | (nk[i] << PIC_CELL_BITS));
          x[i] = x[i] - c;
        }
      });
      gather_by_id(live_by_id(cell.data(), id.data(), n), cell.data(), x.data(), vx.data(), vy.data(), vz.data(),
                   out[s]);
    }
  }
  return PIC_OK;
}

// The live neutrals (FP32 buffer a, extent n) in ascending id order.
int fetch_neutrals(pic_handle* h, const Species32& a, size_t n, HostParticles& o) {
  std::vector<int32_t> cell(n);
  std::vector<float> f(n), vx(n), vy(n), vz(n);
  std::vector<uint64_t> id(n);
  CK(cudaMemcpy(cell.data(), a.cell, n * 4, cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(f.data(), a.frac, n * 4, cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(vx.data(), a.vx, n * 4, cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(vy.data(), a.vy, n * 4, cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(vz.data(), a.vz, n * 4, cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(id.data(), a.id, n * 8, cudaMemcpyDeviceToHost));
  (void)h;
  gather_by_id(live_by_id(cell.data(), id.data(), n), cell.data(), f.data(), vx.data(), vy.data(), vz.data(), o);
  return PIC_OK;
}

template <class T>
void put(std::vector<unsigned char>& b, const T& v) {
  const unsigned char* p = reinterpret_cast<const unsigned char*>(&v);
  b.insert(b.end(), p, p + sizeof(T));
}

template <class T>
void put_arr(std::vector<unsigned char>& b, const std::vector<T>& v) {
  const unsigned char* p = reinterpret_cast<const unsigned char*>(v.data());
  b.insert(b.end(), p, p + sizeof(T) * v.size());
}

// The blob's record groups (charged species 0 and 1, the neutrals): byte offsets and counts; over:
// more records than the handle's capacity (reported as PIC_EOVERFLOW once the blob has passed the
// checks of its contents, so that a damaged blob is always PIC_ECORRUPT).
struct BlobGroups {
  size_t off[3];
  uint64_t n[3];
  bool over;
};

// Every check of a blob that reads only its header: magic, version, configuration hash, counts and
// length; fills the record groups.
int check_header(const pic_handle* h, const unsigned char* b, size_t len, BlobGroups* g) {
  if (len < kHdr + 4 || std::memcmp(b, "PICMCSN1", 8) != 0) return PIC_ECORRUPT;
  uint32_t ver;
  uint64_t hash, step, n[2];
  std::memcpy(&ver, b + 8, 4);
  std::memcpy(&hash, b + 16, 8);
  std::memcpy(&step, b + 24, 8);
  std::memcpy(n, b + 32, 16);
  if (ver != (h->cap_nt ? 4u : 3u) || hash != config_hash(h->cfg)) return PIC_ECORRUPT;
  if (n[0] > (1ull << 40) || n[1] > (1ull << 40)) return PIC_ECORRUPT;
  const size_t charged = kHdr + 44 * (size_t)(n[0] + n[1]);
  uint64_t nn = 0;
  if (ver == 4) {  // the neutral block: u64 n, u64 counters[6], records
    if (len < charged + kNtHdr + 4) return PIC_ECORRUPT;
    std::memcpy(&nn, b + charged, 8);
    if (nn > (1ull << 40) || len != charged + kNtHdr + 44 * nn + 4) return PIC_ECORRUPT;
  } else if (len != charged + 4) {
    return PIC_ECORRUPT;
  }
  g->over = round_up4(nn) > h->cap_nt;
  for (int s = 0; s < 2; ++s) g->over = g->over || round_up4(n[s]) > h->cap[s];
  g->off[0] = kHdr;
  g->off[1] = kHdr + 44 * (size_t)n[0];
  g->off[2] = charged + kNtHdr;
  g->n[0] = n[0];
  g->n[1] = n[1];
  g->n[2] = nn;
  return PIC_OK;
}

// The checks that read the whole blob, on host threads: the CRC, and the range of every cell,
// countdown and fraction.  The cell word is cell | k << 18 | c << 30; a species with the
// null-collision test may leave the countdown pair (k | c << 12) at 0 ("not drawn": the restore
// draws it), else 1 <= k <= 4095; every other species (the neutrals included) carries 0 there.
int check_body(const pic_handle* h, const unsigned char* b, size_t len, const BlobGroups& g) {
  uint32_t crc;
  std::memcpy(&crc, b + len - 4, 4);
  if (crc != crc32_ieee(b, len - 4)) return PIC_ECORRUPT;
  const int N = h->N;
  {
    const size_t* offs = g.off;
    const uint64_t* counts = g.n;
    bool bad = false;
    for (int s = 0; s < 3; ++s) {
      const bool mcc = s < 2 && ((h->ph.mcc_mask >> s) & 1u);
      const size_t m = (size_t)counts[s];
      const unsigned char* cell = b + offs[s];
      const unsigned char* frac = cell + 4 * m;
      const int T = host_threads(12 * m);
      std::vector<char> flag(T, 0);
      std::vector<std::thread> th;
      const size_t chunk = (m + T - 1) / T;
      for (int k = 0; k < T; ++k) {
        th.emplace_back([&, k]() {
          const size_t i0 = std::min(m, (size_t)k * chunk), i1 = std::min(m, i0 + chunk);
          for (size_t i = i0; i < i1; ++i) {
            uint32_t w;
            double f;
            std::memcpy(&w, cell + 4 * i, 4);
            std::memcpy(&f, frac + 8 * i, 8);
            const uint32_t pair = w >> PIC_CELL_BITS;
            const bool pair_ok = mcc ? (pair == 0u || (pair <= (PIC_NEXT_CAND | PIC_NEXT_KMAX) &&
                                                       (pair & PIC_NEXT_KMAX) != 0u))
                                     : pair == 0u;
            if ((int)(w & PIC_CELL_MASK) >= N || !pair_ok || !(f >= 0.0 && f < 1.0)) {
              flag[k] = 1;
              break;
            }
          }
        });
      }
      for (auto& t : th) t.join();
      for (char f : flag) bad = bad || f;
    }
    if (bad) return PIC_ECORRUPT;
  }
  return PIC_OK;
}

int check_blob(const pic_handle* h, const void* buf, size_t len) {
  if (!h || !buf) return PIC_EINVAL;
  const unsigned char* b = static_cast<const unsigned char*>(buf);
  BlobGroups g;
  int rc = check_header(h, b, len, &g);
  if (rc == PIC_OK) rc = check_body(h, b, len, g);
  return rc != PIC_OK ? rc : (g.over ? PIC_EOVERFLOW : PIC_OK);
}

// The same checks as check_body on the device, for a large blob of the FP32 path: the blob is
// copied once into a temporary device buffer (cudaMallocAsync), where k_blob_crc checksums its
// 64 KB blocks and k_blob_ranges checks the records; the host joins the block checksums (the
// operator Z^65536 as four byte tables) and finishes the tail.  On success *dev holds the copy,
// from which the restore then reads; PIC_ECORRUPT frees it.  Returns -1 (nothing allocated)
// when the device path does not apply or the allocation fails: the caller checks on the host.
int check_body_device(pic_handle* h, const unsigned char* b, size_t len, const BlobGroups& g, unsigned char** dev) {
  *dev = nullptr;
  if (h->plain || len < (size_t(16) << 20)) return -1;
  const size_t n = len - 4;
  const size_t nblk = n / 65536;
  const size_t alen = (len + 255) & ~size_t(255);
  const size_t blen = (4 * nblk + 255) & ~size_t(255);
  std::vector<uint32_t> hb(nblk);  // (before the allocation: a failure here frees nothing)
  unsigned char* d = nullptr;
  if (cudaMallocAsync(reinterpret_cast<void**>(&d), alen + blen + 256, h->st) != cudaSuccess) {
    cudaGetLastError();
    return -1;
  }
  uint32_t* blk = reinterpret_cast<uint32_t*>(d + alen);
  unsigned int* bad = reinterpret_cast<unsigned int*>(d + alen + blen);
  // operators: one zero byte, then squared up to 2^16 zero bytes
  Gf2 z;
  z.m[0] = 0xEDB88320u;
  for (int i = 1; i < 32; ++i) z.m[i] = 1u << (i - 1);
  z = gf2_square(gf2_square(gf2_square(z)));
  BlobCrcOps ops;
  for (int k = 0; k < 11; ++k) z = gf2_square(z);  // 2048 bytes
  for (int k = 0; k < 5; ++k) {
    std::memcpy(ops.z[k], z.m, sizeof(z.m));
    z = gf2_square(z);
  }  // z: 65536 bytes
  unsigned int hbad = 0;
  cudaError_t e = cudaMemsetAsync(bad, 0, 4, h->st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d, b, len, cudaMemcpyHostToDevice, h->st);
  if (e == cudaSuccess) e = launch_blob_crc(d, nblk, ops, blk, h->st);
  for (int s = 0; s < 3 && e == cudaSuccess; ++s)
    e = launch_blob_ranges(d + g.off[s], d + g.off[s] + 4 * g.n[s], g.n[s], h->N,
                           s < 2 && ((h->ph.mcc_mask >> s) & 1u) ? 1 : 0, bad, h->st);
  if (e == cudaSuccess && nblk) e = cudaMemcpyAsync(hb.data(), blk, 4 * nblk, cudaMemcpyDeviceToHost, h->st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&hbad, bad, 4, cudaMemcpyDeviceToHost, h->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->st);
  if (e != cudaSuccess) {
    cudaFreeAsync(d, h->st);
    return PIC_ECUDA;
  }
  uint32_t tab[4][256];
  for (int j = 0; j < 4; ++j)
    for (uint32_t x = 0; x < 256; ++x) tab[j][x] = gf2_apply(z, x << (8 * j));
  uint32_t reg = 0xFFFFFFFFu;
  for (size_t i = 0; i < nblk; ++i)
    reg = (tab[0][reg & 0xFFu] ^ tab[1][(reg >> 8) & 0xFFu] ^ tab[2][(reg >> 16) & 0xFFu] ^ tab[3][reg >> 24]) ^ hb[i];
  reg = crc_raw(crc_tables(), reg, b + 65536 * nblk, n - 65536 * nblk);
  uint32_t crc;
  std::memcpy(&crc, b + n, 4);
  if ((reg ^ 0xFFFFFFFFu) != crc || hbad) {
    cudaFreeAsync(d, h->st);
    return PIC_ECORRUPT;
  }
  *dev = d;
  return PIC_OK;
}

int restore_state(pic_handle* h, const void* buf, size_t len, bool checked) {
  if (!h || !buf) return PIC_EINVAL;
  const unsigned char* b = static_cast<const unsigned char*>(buf);
  unsigned char* dev = nullptr;  // a device copy of the blob (large FP32 blobs): uploads read it
  if (!checked) {
    BlobGroups g;
    int rc = check_header(h, b, len, &g);
    if (rc != PIC_OK) return rc;
    if (!g.over) rc = check_body_device(h, b, len, g, &dev);
    if (g.over || rc < 0) rc = check_body(h, b, len, g);
    if (rc == PIC_OK && g.over) rc = PIC_EOVERFLOW;
    if (rc != PIC_OK) {
      if (dev) cudaFreeAsync(dev, h->st);
      return rc;
    }
  }
  struct DevFree {  // the device copy is released however the restore ends
    unsigned char* p;
    cudaStream_t st;
    ~DevFree() {
      if (p) {
        cudaStreamSynchronize(st);
        cudaFreeAsync(p, st);
      }
    }
  } dev_free{dev, h->st};
  uint64_t step, n[2];
  std::memcpy(&step, b + 24, 8);
  std::memcpy(n, b + 32, 16);
  CK(cudaStreamSynchronize(h->st));
  uint64_t cnt[17];
  int64_t wall_charge;
  double wall_energy[2];
  std::memcpy(cnt, b + 48, sizeof(cnt));
  std::memcpy(&wall_charge, b + 48 + 136, 8);
  std::memcpy(wall_energy, b + 48 + 144, 16);
  const int N = h->N;
  const double dx = h->cfg.L / N;
  size_t off = kHdr;
  h->cur = 0;
  // FP32: a species' arrays (m records at blob offset o) go straight to device staging (the sort's
  // second buffer, unused between sorts) and a kernel converts them into dst
  auto upload32 = [&](size_t o, size_t m, const Species32& dstsp, int species) -> int {
    char* stage = h->stage;
    const size_t stage_bytes = h->stage_bytes;
    const size_t per = std::max<size_t>(4, (stage_bytes - 6 * 256) / 44 / 4 * 4);
    const unsigned char* sb = dev ? dev : b;  // the device copy when there is one
    const cudaMemcpyKind kind = dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    const unsigned char* src[6] = {sb + o, sb + o + 4 * m, sb + o + 12 * m, sb + o + 20 * m, sb + o + 28 * m,
                                   sb + o + 36 * m};
    const size_t width[6] = {4, 8, 8, 8, 8, 8};
    for (size_t done = 0; done < m; done += per) {
      const size_t cnt_i = std::min(per, m - done);
      char* dst[6];
      size_t so = 0;
      for (int a = 0; a < 6; ++a) {
        dst[a] = stage + so;
        so += (width[a] * cnt_i + 255) & ~size_t(255);
        CK(cudaMemcpyAsync(dst[a], src[a] + width[a] * done, width[a] * cnt_i, kind, h->st));
      }
      CK(launch_restore32(reinterpret_cast<const int*>(dst[0]), reinterpret_cast<const double*>(dst[1]),
                          reinterpret_cast<const double*>(dst[2]), reinterpret_cast<const double*>(dst[3]),
                          reinterpret_cast<const double*>(dst[4]), reinterpret_cast<const unsigned long long*>(dst[5]),
                          cnt_i, dstsp, done, h->ph, species, step, h->st));
    }
    const size_t mp = (size_t)round_up4(m);
    if (mp > m) {
      const int dead[4] = {PIC_DEAD_CELL, PIC_DEAD_CELL, PIC_DEAD_CELL, PIC_DEAD_CELL};
      CK(cudaMemcpyAsync(dstsp.cell + m, dead, 4 * (mp - m), cudaMemcpyHostToDevice, h->st));
    }
    CK(cudaStreamSynchronize(h->st));
    return PIC_OK;
  };
  for (int s = 0; s < 2; ++s) {
    const size_t m = (size_t)n[s];
    const size_t mp = (size_t)round_up4(m);
    if (!h->plain) {
      const int rc = upload32(off, m, h->a32[0][s], s);
      if (rc != PIC_OK) return rc;
    } else {
      std::vector<double> x(mp, -1.0), a1(mp, 0.0), a2(mp, 0.0), a3(mp, 0.0);
      std::vector<uint64_t> id2(mp, 0ull);
      std::vector<unsigned> nk(mp, 0u);
      const unsigned char* cell = b + off;
      for (size_t i = 0; i < m; ++i) {
        uint32_t w;
        double f;
        std::memcpy(&w, cell + 4 * i, 4);
        std::memcpy(&f, cell + 4 * m + 8 * i, 8);
        const int32_t c = (int32_t)(w & PIC_CELL_MASK);
        nk[i] = w >> PIC_CELL_BITS;
        double xx = (double)c + f;
        if (xx >= (double)c + 1.0) xx = std::nextafter((double)c + 1.0, 0.0);
        x[i] = xx;
        std::memcpy(&a1[i], cell + 12 * m + 8 * i, 8);
        std::memcpy(&a2[i], cell + 20 * m + 8 * i, 8);
        std::memcpy(&a3[i], cell + 28 * m + 8 * i, 8);
        std::memcpy(&id2[i], cell + 36 * m + 8 * i, 8);
      }
      const Species64& a = h->a64[s];
      CK(cudaMemcpy(a.x, x.data(), 8 * mp, cudaMemcpyHostToDevice));
      CK(cudaMemcpy(a.vx, a1.data(), 8 * mp, cudaMemcpyHostToDevice));
      CK(cudaMemcpy(a.vy, a2.data(), 8 * mp, cudaMemcpyHostToDevice));
      CK(cudaMemcpy(a.vz, a3.data(), 8 * mp, cudaMemcpyHostToDevice));
      CK(cudaMemcpy(a.id, id2.data(), 8 * mp, cudaMemcpyHostToDevice));
      CK(cudaMemcpy(a.nk, nk.data(), 4 * mp, cudaMemcpyHostToDevice));
      CK(launch_fill_pairs64(a.nk, a.id, m, h->ph, s, step, h->st));  // pairs the blob left undrawn
    }
    off += 44 * m;
  }
  CK(cudaStreamSynchronize(h->st));
  Ctl c;
  std::memset(&c, 0, sizeof(c));
  for (int s = 0; s < 2; ++s) {
    c.n_cur[s] = round_up4(n[s]);
    c.n_live[s] = n[s];
  }
  if (h->cap_nt) {  // version 2: the neutral block follows the charged records (off is past them)
    uint64_t nn, nc[6];
    std::memcpy(&nn, b + off, 8);
    std::memcpy(nc, b + off + 8, sizeof(nc));
    const int rc = upload32(off + kNtHdr, (size_t)nn, h->nt[0], 2);
    if (rc != PIC_OK) return rc;
    h->nt_buf = 0;
    c.nt_cur = round_up4(nn);
    c.nt_live = nn;
    c.nt_recycled[0] = nc[0];
    c.nt_recycled[1] = nc[1];
    c.nt_lost[0] = nc[2];
    c.nt_lost[1] = nc[3];
    c.nt_ionized = nc[4];
    c.nt_near = nc[5];
  }
  int k = 0;
  for (int s = 0; s < 2; ++s)
    for (int side = 0; side < 2; ++side) c.wall_hits[s][side] = cnt[k++];
  for (int i = 0; i < 5; ++i) c.coll[i] = cnt[k++];
  for (int s = 0; s < 2; ++s) c.near_thr[s] = cnt[k++];
  for (int s = 0; s < 2; ++s) c.viol[s] = cnt[k++];
  for (int s = 0; s < 2; ++s) c.births[s] = cnt[k++];
  c.source_pairs = cnt[k++];
  c.dropped = cnt[k++];
  c.wall_charge = wall_charge;
  for (int s = 0; s < 2; ++s) {
    const double w = dx / h->cfg.ppc[s];
    c.wall_energy_fx[s] = (unsigned long long)std::llrint(wall_energy[s] / w * 16777216.0);
  }
  CK(cudaMemcpy(h->ctl, &c, sizeof(c), cudaMemcpyHostToDevice));
  // clear the grid accumulators (a previous step may have left counts for a sort)
  if (!h->plain) {
    for (int s = 0; s < 2; ++s) {
      CK(cudaMemsetAsync(h->cnt[s], 0, sizeof(unsigned int) * N, h->st));
      CK(cudaMemsetAsync(h->S[s], 0, sizeof(unsigned long long) * N, h->st));
    }
  } else {
    for (int s = 0; s < 2; ++s) CK(cudaMemsetAsync(h->acc[s], 0, sizeof(double) * (N + 1), h->st));
  }
  h->step = step;
  return PIC_OK;
}

// The particle phase of one step: the particle, neutral and source kernels (the deposit goes into
// the per-cell counts); records in h whether the step sorts and whether it moved the particles.
int step_particles(pic_handle* h) {
  const bool sort_now = !h->plain && (h->step % (unsigned long long)h->cfg.sort_interval) == 0ull;
  const bool scatter = !h->plain && h->pending_scatter;
  EvPair e;
  if (!h->plain) {
    StepParams32 P = params32(h);
    const bool sum_ke = h->ke_every > 0 && ((h->step + 1) % (unsigned long long)h->ke_every) == 0ull;
    P.sum_ke = sum_ke ? 1u : 0u;
    h->ke_valid = sum_ke;
    if (scatter) {  // the step after a sort: read buffer cur, fill buffer 1 - cur in sorted order
      for (int s = 0; s < 2; ++s) P.sp[s] = h->a32[1 - h->cur][s];
      P.scatter = 1u;
    }
    prof_begin(h, scatter ? K_STEP_SCATTER : K_STEP, &e);
    // both read buffer cur
    if (!h->maps_ok) return PIC_ECUDA;
    CK(scatter ? launch_step32_scatter(P, h->maps[h->cur], h->grid_scatter, h->st)
               : launch_step32(P, h->maps[h->cur], h->grid_step, h->st));
    prof_end(h, &e);
    if (h->cap_nt) {  // the neutrals alive at the step start, and the ions recycled in this step:
      // in place, or compacted into the other buffer on the steps that sort
      NeutralParams Q = neutral_params(h, P);
      if (!sort_now) Q.dst = Q.src;
      prof_begin(h, sort_now ? K_NEUTRAL_COMPACT : K_NEUTRAL, &e);
      CK(launch_neutral32(Q, sort_now, h->grid_neutral, h->st));
      prof_end(h, &e);
    }
    if (h->cfg.source_mode == PIC_SOURCE_PAIRS) {
      prof_begin(h, K_SOURCE, &e);
      CK(launch_source32(P, h->st));
      prof_end(h, &e);
    }
    if (scatter) {
      h->cur = 1 - h->cur;
      h->pending_scatter = false;
    }
  } else {
    const StepParams64 P = params64(h);
    prof_begin(h, K_STEP, &e);
    CK(launch_step64(P, h->grid_step, h->st));
    prof_end(h, &e);
    if (h->cfg.source_mode == PIC_SOURCE_PAIRS) {
      prof_begin(h, K_SOURCE, &e);
      CK(launch_source64(P, h->st));
      prof_end(h, &e);
    }
  }
  h->open_sort = sort_now;
  h->open_scatter = scatter;
  return PIC_OK;
}

// The rest of the step: field solve (of this handle's deposits, or of the deposits R_total of a
// decomposed simulation), bookkeeping, and the sort scan on sort steps; the step count advances.
int step_close(pic_handle* h, const long long* R_total) {
  EvPair e;
  const bool sort_now = h->open_sort, scatter = h->open_scatter;
  prof_begin(h, K_FIELD, &e);
  PoissonParams F = field_params(h, sort_now, true);
  F.scatter_step = scatter ? 1 : 0;
  F.R_in = R_total;
  if (h->cap_nt) {  // the buffer the neutral step wrote
    F.nt_pad = h->nt[sort_now ? 1 - h->nt_buf : h->nt_buf];
    F.nt_append = sort_now ? 0 : 1;
  }
  CK(launch_field(F, h->st));
  prof_end(h, &e);
  if (h->cap_nt && sort_now) h->nt_buf = 1 - h->nt_buf;
  if (sort_now) {
    // the counting sort: cursors from this step's counts now; the particles move during the next
    // step (k_step32 in scatter mode), which saves a read and a write of every particle
    prof_begin(h, K_SORT, &e);
    Species32 src[2] = {h->a32[h->cur][0], h->a32[h->cur][1]};
    Species32 dst[2] = {h->a32[1 - h->cur][0], h->a32[1 - h->cur][1]};
    CK(launch_sort_scan32(src, dst, h->cnt, h->cursor, h->cap, h->ctl, h->N, h->st));
    prof_end(h, &e);
    h->pending_scatter = true;
  }
  h->step += 1;
  return PIC_OK;
}

// Particle decomposition needs the FP32 path and the integer-exact field (an exact sum of the
// parts' deposits), and none of the per-step inputs a part could not draw alone (pair source ids,
// tracked neutrals).
bool split_ok(const pic_handle* h) {
  return !h->plain && exact_possible(h->cfg) && h->cfg.source_mode == PIC_SOURCE_NONE && !h->cap_nt;
}

bool blob_step(const void* buf, size_t len, unsigned long long* step) {
  if (!buf || len < kHdr + 4 || std::memcmp(buf, "PICMCSN1", 8) != 0) return false;
  uint64_t v;
  std::memcpy(&v, static_cast<const unsigned char*>(buf) + 24, 8);
  *step = v;
  return true;
}

}  // namespace picx

using namespace picx;

// =============================================================================================
extern "C" {

uint32_t pic_blob_crc32(const void* p, size_t n) {
  if (!p || !n) return 0u;
  try {
      return crc32_ieee(static_cast<const unsigned char*>(p), n);
    } catch (...) {  // no helper thread could start: the same CRC on this thread
      return crc32_serial(static_cast<const unsigned char*>(p), n);
    }
  }

  const char* pic_strerror(int status) {
    switch (status) {
      case PIC_OK: return "ok";
      case PIC_EINVAL: return "invalid argument or configuration";
      case PIC_ENOMEM: return "out of memory or workspace too small";
      case PIC_ECUDA: return "CUDA runtime error";
      case PIC_EOVERFLOW: return "particle capacity exceeded";
      case PIC_ECORRUPT: return "corrupt or mismatched snapshot";
      case PIC_ETIMEOUT: return "device wait timed out";
      case PIC_EDEVICE: return "device-side check failed";
      default: return "unknown status";
    }
  }

  int pic_workspace_size(const pic_config* cfg, size_t* bytes) {
    PIC_ENTRY_TRY
    if (!valid(cfg) || !bytes) return PIC_EINVAL;
    pic_handle tmp;
    tmp.cfg = *cfg;
    tmp.N = cfg->ncells;
    tmp.plain = cfg->precision == PIC_FP64_PLAIN;
    for (int s = 0; s < 2; ++s) tmp.cap[s] = capacity(cfg, s);
    tmp.cap_nt = neutral_capacity(cfg);
    layout(&tmp, nullptr, bytes);
    return PIC_OK;
    PIC_ENTRY_CATCH
  }

  int pic_init(const pic_config* cfg, void* workspace, size_t workspace_bytes, void* cuda_stream, pic_handle** out) {
    PIC_ENTRY_TRY
    if (!out) return PIC_EINVAL;
    *out = nullptr;
    if (!valid(cfg)) return PIC_EINVAL;
    if (workspace && (reinterpret_cast<uintptr_t>(workspace) & 255u)) return PIC_EINVAL;
    pic_handle* h = new (std::nothrow) pic_handle();
    if (!h) return PIC_ENOMEM;
  try {
    h->cfg = *cfg;
    h->st = static_cast<cudaStream_t>(cuda_stream);
    h->N = cfg->ncells;
    h->plain = cfg->precision == PIC_FP64_PLAIN;
    for (int s = 0; s < 2; ++s) h->cap[s] = capacity(cfg, s);
    h->cap_nt = neutral_capacity(cfg);
    size_t need = 0;
    layout(h, nullptr, &need);
    if (workspace) {
      if (workspace_bytes < need) {
        delete h;
        return PIC_ENOMEM;
      }
      h->ws = workspace;
    } else {
      if (cudaMalloc(&h->ws, need) != cudaSuccess) {
        delete h;
        return PIC_ENOMEM;
      }
      h->owns_ws = true;
    }
    h->ws_bytes = need;
    layout(h, static_cast<char*>(h->ws), &need);
    derive(h);
    if (!h->plain && make_step_maps(h) != PIC_OK) {
      if (h->owns_ws) cudaFree(h->ws);
      delete h;
      return PIC_ECUDA;
    }
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 152;
    h->grid_step = sms * (h->plain ? occupancy_step64() : occupancy_step32());
    h->grid_scatter = h->plain ? 0 : sms * occupancy_step32(true);
    {  // small runs: no more CTAs than the particle capacity can keep busy (a warp per chunk of
       // 128 particles, a thread per particle on the plain path); large runs fill every SM
      const unsigned long long room = h->cap[0] + h->cap[1];
      const unsigned long long need = h->plain ? (room + 255) / 256 : (room + PIC_TILE - 1) / PIC_TILE;
      const int cap_grid = (int)std::max<unsigned long long>(1ull, std::min<unsigned long long>(need, 1ull << 20));
      h->grid_step = std::min(h->grid_step, cap_grid);
      if (!h->plain) h->grid_scatter = std::min(h->grid_scatter, cap_grid);
    }
    if (!h->plain && h->fgrid) {  // the grid-wide field solve: a CTA per 256 nodes, at most one per SM
      const int want = (h->N + 1 + 255) / 256;
      h->field_ctas = std::max(1, std::min(std::min(want, sms), PIC_FIELD_GRID_MAX));
    }
    h->grid_sort = sms * 16;
    h->grid_diag = sms * 8;
    h->grid_neutral = h->cap_nt ? sms * occupancy_neutral32() : 0;
    *out = h;

    int rc = PIC_OK;
    // zero the grid arrays and the control block (particle arrays are written by the load)
    const char* grid_begin = reinterpret_cast<const char*>(h->plain ? (void*)h->acc[0] : (void*)h->cnt[0]);
    size_t grid_off = (size_t)(grid_begin - static_cast<char*>(h->ws));
    if (cudaMemsetAsync(static_cast<char*>(h->ws) + grid_off, 0, need - 256 - grid_off, h->st) != cudaSuccess ||
        cudaMemsetAsync(h->ctl, 0, sizeof(Ctl), h->st) != cudaSuccess) {
      rc = PIC_ECUDA;
    }
    if (rc == PIC_OK) rc = load_initial(h);
    if (rc != PIC_OK) {
      pic_free(h);
      *out = nullptr;
    }
    return rc;
  } catch (...) {  // a host allocation or thread failed part way: release what was taken
    pic_free(h);
    *out = nullptr;
    return PIC_ENOMEM;
  }
  PIC_ENTRY_CATCH
}

int pic_step(pic_handle* h, int32_t n) {
  PIC_ENTRY_TRY
  if (!h || n < 0 || h->split_open) return PIC_EINVAL;
  for (int32_t k = 0; k < n; ++k) {
    int rc = step_particles(h);
    if (rc == PIC_OK) rc = step_close(h, nullptr);
    if (rc != PIC_OK) return rc;
  }
  return PIC_OK;
  PIC_ENTRY_CATCH
}

size_t pic_diag_bytes(void) { return sizeof(Ctl); }

int pic_set_diag_interval(pic_handle* h, int32_t every) {
  PIC_ENTRY_TRY
  if (!h || every < 0) return PIC_EINVAL;
  h->ke_every = every;
  return PIC_OK;
  PIC_ENTRY_CATCH
}

int pic_keep_subset(pic_handle* h, uint32_t part, uint32_t nparts) {
  PIC_ENTRY_TRY
  if (!h || !split_ok(h) || h->split_open || nparts < 1 || part >= nparts) return PIC_EINVAL;
  int rc = check_errors(h);
  if (rc != PIC_OK) return rc;
  CK(launch_keep_subset(h->a32[h->cur][0], h->a32[h->cur][1], h->ctl, part, nparts, h->st));
  rc = refresh_field(h);  // deposit of the part's particles, its own field, full sort + compaction
  if (rc == PIC_OK) rc = check_errors(h);
  if (rc != PIC_OK) return rc;
  if (part != 0) {  // cumulative counters and sums stay with part 0, so that the parts add up
    Ctl c;
    CK(cudaMemcpy(&c, h->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost));
    std::memset(c.wall_hits, 0, sizeof(c.wall_hits));
    std::memset(c.coll, 0, sizeof(c.coll));
    std::memset(c.near_thr, 0, sizeof(c.near_thr));
    std::memset(c.viol, 0, sizeof(c.viol));
    std::memset(c.births, 0, sizeof(c.births));
    std::memset(c.wall_energy_fx, 0, sizeof(c.wall_energy_fx));
    c.source_pairs = c.dropped = 0ull;
    c.wall_charge = 0;
    c.particle_steps = 0ull;
    CK(cudaMemcpy(h->ctl, &c, sizeof(Ctl), cudaMemcpyHostToDevice));
  }
  return PIC_OK;
  PIC_ENTRY_CATCH
}

int pic_local_deposit(pic_handle* h, int64_t* R_local) {
  PIC_ENTRY_TRY
  if (!h || !R_local || !split_ok(h) || h->split_open) return PIC_EINVAL;
  // a deposit pass over the particles as they stand (no push, no collision), the node deposits,
  // then the per-cell accumulators cleared again
  Phys saved = h->ph;
  h->ph.push_mask = 0u;
  h->ph.coll_mask = 0u;
  h->ph.mcc_mask = 0u;
  StepParams32 P = params32(h);
  h->ph = saved;
  if (!h->maps_ok) return PIC_ECUDA;
  CK(launch_step32(P, h->maps[h->cur], h->grid_step, h->st));
  const PoissonParams F = field_params(h, false, false);
  CK(launch_node_deposit(F, reinterpret_cast<long long*>(R_local), h->st));
  for (int s = 0; s < 2; ++s) {
    CK(cudaMemsetAsync(h->cnt[s], 0, sizeof(unsigned int) * h->N, h->st));
    CK(cudaMemsetAsync(h->S[s], 0, sizeof(unsigned long long) * h->N, h->st));
  }
  return PIC_OK;
  PIC_ENTRY_CATCH
}

int pic_solve_deposit(pic_handle* h, const int64_t* R_total) {
  PIC_ENTRY_TRY
  if (!h || !R_total || !split_ok(h) || h->split_open) return PIC_EINVAL;
  PoissonParams F = field_params(h, true, false);
  F.R_in = reinterpret_cast<const long long*>(R_total);
  F.no_book = 1;
  CK(launch_field(F, h->st));
  return PIC_OK;
  PIC_ENTRY_CATCH
}

int pic_step_begin(pic_handle* h, int64_t* R_local) {
  PIC_ENTRY_TRY
  if (!h || !R_local || !split_ok(h) || h->split_open) return PIC_EINVAL;
  int rc = step_particles(h);
  if (rc != PIC_OK) return rc;
  const PoissonParams F = field_params(h, false, false);
  CK(launch_node_deposit(F, reinterpret_cast<long long*>(R_local), h->st));
  h->split_open = true;
  return PIC_OK;
  PIC_ENTRY_CATCH
}

int pic_step_end(pic_handle* h, const int64_t* R_total) {
  PIC_ENTRY_TRY
  if (!h || !R_total || !h->split_open) return PIC_EINVAL;
  h->split_open = false;
  return step_close(h, reinterpret_cast<const long long*>(R_total));
  PIC_ENTRY_CATCH
}

int pic_sync(pic_handle* h) {
  PIC_ENTRY_TRY
  if (!h) return PIC_EINVAL;
  return check_errors(h);
  PIC_ENTRY_CATCH
}

int pic_diag_async(pic_handle* h, void* host_buf, uint32_t what) {
  PIC_ENTRY_TRY
  if (!h || !host_buf || what > PIC_DIAG_COUNTERS) return PIC_EINVAL;
  EvPair e;
  prof_begin(h, K_DIAG, &e);
  CK(launch_store_u64(&h->ctl->diag_step, h->step, h->st));
  CK(launch_store_u64(&h->ctl->diag_what, what, h->st));
  if (what == PIC_DIAG_COUNTERS) {
    prof_end(h, &e);
    CK(cudaMemcpyAsync(host_buf, h->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, h->st));
    return PIC_OK;
  }
  CK(cudaMemsetAsync(&h->ctl->netq, 0, sizeof(h->ctl->netq), h->st));
  // kinetic energy into ke_fx: the last step's sum when it made one (FP32 path, ke_last), else one
  // reduction pass here (same fixed point, same bits)
  if (!h->plain && h->ke_valid) {
    CK(cudaMemcpyAsync(h->ctl->ke_fx, h->ctl->ke_last, sizeof(h->ctl->ke_fx), cudaMemcpyDeviceToDevice, h->st));
  } else {
    CK(cudaMemsetAsync(h->ctl->ke_fx, 0, sizeof(h->ctl->ke_fx), h->st));
    if (h->plain)
      CK(launch_diag64(params64(h), h->grid_diag, h->st));
    else
      CK(launch_diag32(params32(h), h->grid_diag, h->st));
  }
  CK(launch_diag_grid(h->R[0], h->R[1], h->cfg.charge[0] > 0 ? 1 : -1, h->cfg.charge[1] > 0 ? 1 : -1, h->E, h->N,
                      h->cfg.L / h->N, h->ctl, h->st));
  prof_end(h, &e);
  CK(cudaMemcpyAsync(host_buf, h->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, h->st));
  return PIC_OK;
  PIC_ENTRY_CATCH
}

int pic_diag_decode(const pic_handle* h, const void* host_buf, pic_diag_t* d) {
  PIC_ENTRY_TRY
  if (!h || !host_buf || !d) return PIC_EINVAL;
  Ctl c;
  std::memcpy(&c, host_buf, sizeof(Ctl));
  const int rc = status_of(c.error);
  if (rc != PIC_OK) return rc;
  const int N = h->N;
  std::memset(d, 0, sizeof(*d));
  const double dx = h->cfg.L / N;
  const bool all = c.diag_what == PIC_DIAG_ALL;
  d->step = c.diag_step;
  for (int s = 0; s < 2; ++s) {
    const double w = dx / h->cfg.ppc[s];
    d->n[s] = c.n_live[s];
    d->wall_hits[s][0] = c.wall_hits[s][0];
    d->wall_hits[s][1] = c.wall_hits[s][1];
    d->near_threshold[s] = c.near_thr[s];
    d->nu_max_violations[s] = c.viol[s];
    d->births[s] = c.births[s];
    d->ke[s] = all ? (double)c.ke_fx[s] * (1.0 / 16777216.0) * w : 0.0;
    d->wall_energy[s] = (double)c.wall_energy_fx[s] * (1.0 / 16777216.0) * w;
  }
  for (int k = 0; k < 5; ++k) d->coll[k] = c.coll[k];
  d->source_pairs = c.source_pairs;
  d->dropped = c.dropped;
  d->wall_charge = c.wall_charge;
  d->particle_steps = c.particle_steps;
  if (all) {
    d->net_charge_units = c.netq;
    double fe = 0.0;
    for (int b = 0; b < PIC_DIAG_BLOCKS; ++b) fe += c.fe_part[b];
    d->field_energy = fe;
  }
  return PIC_OK;
  PIC_ENTRY_CATCH
}

int pic_diag(pic_handle* h, pic_diag_t* d) {
  PIC_ENTRY_TRY
  if (!h || !d) return PIC_EINVAL;
  // one device-to-host read of the control block (its error word included) and one wait
  Ctl c;
  int rc = pic_diag_async(h, &c, PIC_DIAG_ALL);
  if (rc != PIC_OK) return rc;
  CK(cudaStreamSynchronize(h->st));
  return pic_diag_decode(h, &c, d);
  PIC_ENTRY_CATCH
}

int pic_neutral_diag(pic_handle* h, pic_neutral_diag_t* d) {
  PIC_ENTRY_TRY
  if (!h || !d || !h->cap_nt) return PIC_EINVAL;
  CK(cudaMemsetAsync(&h->ctl->nt_ke_fx, 0, sizeof(h->ctl->nt_ke_fx), h->st));
  EvPair e;
  prof_begin(h, K_DIAG, &e);
  CK(launch_ndiag32(h->nt[h->nt_buf], h->ctl, (float)h->cfg.mass[1], h->grid_diag, h->st));
  prof_end(h, &e);
  Ctl c;
  CK(cudaMemcpyAsync(&c, h->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, h->st));
  CK(cudaStreamSynchronize(h->st));
  const int rc = status_of(c.error);
  if (rc != PIC_OK) return rc;
  std::memset(d, 0, sizeof(*d));
  d->n = c.nt_live;
  for (int k = 0; k < 2; ++k) {
    d->recycled[k] = c.nt_recycled[k];
    d->lost[k] = c.nt_lost[k];
  }
  d->ionized = c.nt_ionized;
  d->near_threshold = c.nt_near;
  d->particle_steps = c.nt_particle_steps;
  d->ke = (double)c.nt_ke_fx * (1.0 / 16777216.0) * (h->cfg.L / h->N / h->cfg.ppc[1]);
  return PIC_OK;
  PIC_ENTRY_CATCH
}

int pic_get_field(pic_handle* h, int64_t* R, double* rho, double* phi, float* E, size_t nnodes) {
  PIC_ENTRY_TRY
  if (!h || nnodes != (size_t)h->N + 1) return PIC_EINVAL;
  int rc = check_errors(h);
  if (rc != PIC_OK) return rc;
  rc = field_diagnostics(h);
  if (rc != PIC_OK) return rc;
  CK(cudaStreamSynchronize(h->st));
  if (R) {
    CK(cudaMemcpy(R, h->R[0], sizeof(int64_t) * nnodes, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(R + nnodes, h->R[1], sizeof(int64_t) * nnodes, cudaMemcpyDeviceToHost));
  }
  if (rho) CK(cudaMemcpy(rho, h->rho, sizeof(double) * nnodes, cudaMemcpyDeviceToHost));
  if (phi) CK(cudaMemcpy(phi, h->phi, sizeof(double) * nnodes, cudaMemcpyDeviceToHost));
  if (E) {
    std::vector<double> e(nnodes);
    CK(cudaMemcpy(e.data(), h->E, sizeof(double) * nnodes, cudaMemcpyDeviceToHost));
    for (size_t j = 0; j < nnodes; ++j) E[j] = (float)e[j];
  }
  return PIC_OK;
  PIC_ENTRY_CATCH
}

int pic_storage_order(pic_handle* h, int32_t species, int32_t* cell, uint64_t* ids, size_t cap, size_t* n) {
  PIC_ENTRY_TRY
  if (!h || !n || h->plain || species < 0 || species > 1) return PIC_EINVAL;
  int rc = check_errors(h);
  if (rc != PIC_OK) return rc;
  unsigned long long ext = 0;
  CK(cudaMemcpy(&ext, &h->ctl->n_cur[species], sizeof(ext), cudaMemcpyDeviceToHost));
  *n = (size_t)ext;
  if (!cell && !ids) return PIC_OK;
  if (cap < (size_t)ext) return PIC_ENOMEM;
  const Species32& a = h->a32[h->cur][species];
  if (cell && ext) {
    CK(cudaMemcpy(cell, a.cell, sizeof(int32_t) * ext, cudaMemcpyDeviceToHost));
    for (size_t i = 0; i < (size_t)ext; ++i)  // the cell alone (the word also carries the countdown)
      if (cell[i] != PIC_DEAD_CELL) cell[i] &= PIC_CELL_MASK;
  }
  if (ids && ext) CK(cudaMemcpy(ids, a.id, sizeof(uint64_t) * ext, cudaMemcpyDeviceToHost));
  return PIC_OK;
  PIC_ENTRY_CATCH
}

int pic_snapshot(pic_handle* h, void* buf, size_t cap, size_t* needed) {
  PIC_ENTRY_TRY
  if (!h) return PIC_EINVAL;
  int rc = check_errors(h);
  if (rc != PIC_OK && rc != PIC_EOVERFLOW) return rc;
  // a size query reads only the live counts of the control block and moves no particles (after
  // a neutral overflow the count still includes the neutrals that found no slot: an upper bound)
  Ctl c;
  CK(cudaStreamSynchronize(h->st));
  CK(cudaMemcpy(&c, h->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost));
  if (!buf) {
    if (needed)
      *needed = kHdr + 4 + 44 * (size_t)(c.n_live[0] + c.n_live[1]) +
                (h->cap_nt ? kNtHdr + 44 * (size_t)c.nt_live : 0);
    return PIC_OK;
  }
  HostParticles P[2], NT;
  rc = fetch_particles(h, P, &c);
  if (rc != PIC_OK) return rc;
  if (h->cap_nt) {
    rc = fetch_neutrals(h, h->nt[h->nt_buf], (size_t)c.nt_cur, NT);
    if (rc != PIC_OK) return rc;
  }
  // the blob holds the live entries found in the arrays
  const size_t need = kHdr + 4 + 44 * (P[0].id.size() + P[1].id.size()) + (h->cap_nt ? kNtHdr + 44 * NT.id.size() : 0);
  if (needed) *needed = need;
  if (cap < need) return PIC_EINVAL;
  // header, then each array copied straight into the caller's buffer (host threads for the
  // large ones), then the CRC of everything before it
  unsigned char* const out = static_cast<unsigned char*>(buf);
  size_t at = 0;
  const auto put_raw = [&](const void* src, size_t bytes) {
    if (bytes >= (size_t)(64u << 20)) {
      const unsigned char* p = static_cast<const unsigned char*>(src);
      unsigned char* d = out + at;
      host_parallel(bytes, 2, [&](size_t lo, size_t hi) { std::memcpy(d + lo, p + lo, hi - lo); });
    } else if (bytes) {
      std::memcpy(out + at, src, bytes);
    }
    at += bytes;
  };
  const auto put_u64 = [&](uint64_t v) { put_raw(&v, 8); };
  put_raw("PICMCSN1", 8);
  const uint32_t ver[2] = {(uint32_t)(h->cap_nt ? 4 : 3), 0u};
  put_raw(ver, 8);
  put_u64(config_hash(h->cfg));
  put_u64((uint64_t)h->step);
  put_u64((uint64_t)P[0].id.size());
  put_u64((uint64_t)P[1].id.size());
  for (int s = 0; s < 2; ++s)
    for (int k = 0; k < 2; ++k) put_u64((uint64_t)c.wall_hits[s][k]);
  for (int k = 0; k < 5; ++k) put_u64((uint64_t)c.coll[k]);
  for (int s = 0; s < 2; ++s) put_u64((uint64_t)c.near_thr[s]);
  for (int s = 0; s < 2; ++s) put_u64((uint64_t)c.viol[s]);
  for (int s = 0; s < 2; ++s) put_u64((uint64_t)c.births[s]);
  put_u64((uint64_t)c.source_pairs);
  put_u64((uint64_t)c.dropped);
  const int64_t wall_charge = (int64_t)c.wall_charge;
  put_raw(&wall_charge, 8);
  const double dx = h->cfg.L / h->N;
  for (int s = 0; s < 2; ++s) {
    const double e = (double)c.wall_energy_fx[s] * (1.0 / 16777216.0) * (dx / h->cfg.ppc[s]);
    put_raw(&e, 8);
  }
  const auto put_species = [&](const HostParticles& q) {
    put_raw(q.cell.data(), 4 * q.cell.size());
    put_raw(q.frac.data(), 8 * q.frac.size());
    put_raw(q.vx.data(), 8 * q.vx.size());
    put_raw(q.vy.data(), 8 * q.vy.size());
    put_raw(q.vz.data(), 8 * q.vz.size());
    put_raw(q.id.data(), 8 * q.id.size());
  };
  for (int s = 0; s < 2; ++s) put_species(P[s]);
  if (h->cap_nt) {
    put_u64((uint64_t)NT.id.size());
    for (int k = 0; k < 2; ++k) put_u64((uint64_t)c.nt_recycled[k]);
    for (int k = 0; k < 2; ++k) put_u64((uint64_t)c.nt_lost[k]);
    put_u64((uint64_t)c.nt_ionized);
    put_u64((uint64_t)c.nt_near);
    put_species(NT);
  }
  if (at + 4 != need) return PIC_EDEVICE;
  const uint32_t crc = crc32_ieee(out, at);
  put_raw(&crc, 4);
  return PIC_OK;
  PIC_ENTRY_CATCH
}

int pic_restore(pic_handle* h, const void* buf, size_t len) {
  PIC_ENTRY_TRY
  int rc = restore_state(h, buf, len, false);
  if (rc != PIC_OK) return rc;
  rc = refresh_field(h);
  if (rc != PIC_OK) return rc;
  return check_errors(h);
  PIC_ENTRY_CATCH
}

int pic_profile(pic_handle* h, int enable) {
  PIC_ENTRY_TRY
  if (!h) return PIC_EINVAL;
  if (!enable && h->prof) {
    cudaStreamSynchronize(h->st);
    prof_harvest(h);
  }
  h->prof = enable != 0;
  return PIC_OK;
  PIC_ENTRY_CATCH
}

int pic_kernel_times(pic_handle* h, double* ms, uint64_t* launches, const char** names, int32_t nkinds) {
  PIC_ENTRY_TRY
  if (!h || nkinds < 0) return PIC_EINVAL;
  CK(cudaStreamSynchronize(h->st));
  prof_harvest(h);
  for (int k = 0; k < nkinds && k < PIC_KERNEL_KINDS; ++k) {
    if (ms) ms[k] = h->ms[k];
    if (launches) launches[k] = h->launches[k];
    if (names) names[k] = kKindNames[k];
  }
  for (int k = 0; k < PIC_KERNEL_KINDS; ++k) {
    h->ms[k] = 0.0;
    h->launches[k] = 0;
  }
  return PIC_OK;
  PIC_ENTRY_CATCH
}

void pic_free(pic_handle* h) {
  if (!h) return;
  cudaStreamSynchronize(h->st);
  prof_harvest(h);
  for (cudaEvent_t x : h->ev_free) cudaEventDestroy(x);
  if (h->owns_ws && h->ws) cudaFree(h->ws);
  delete h;
}

int pic_selftest_timeout(void* cuda_stream, double* seconds) {
  PIC_ENTRY_TRY
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  unsigned long long* d = nullptr;
  if (cudaMalloc(&d, 2 * sizeof(unsigned long long)) != cudaSuccess) return PIC_ENOMEM;
  unsigned long long out[2] = {0ull, 0ull};
  cudaError_t e = launch_selftest_wait(d, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(out, d, sizeof(out), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(d);
  if (e != cudaSuccess) return PIC_ECUDA;
  if (seconds) *seconds = (double)out[1] * 1e-9;
  return status_of((unsigned)out[0]);
  PIC_ENTRY_CATCH
}

int pic_philox(const uint32_t* ctr, const uint32_t* key, uint32_t* out, size_t n, void* cuda_stream) {
  PIC_ENTRY_TRY
  if (n && (!ctr || !key || !out)) return PIC_EINVAL;
  if ((reinterpret_cast<uintptr_t>(ctr) & 15u) || (reinterpret_cast<uintptr_t>(out) & 15u) ||
      (reinterpret_cast<uintptr_t>(key) & 7u))
    return PIC_EINVAL;
  return launch_philox(ctr, key, out, n, static_cast<cudaStream_t>(cuda_stream)) == cudaSuccess ? PIC_OK : PIC_ECUDA;
  PIC_ENTRY_CATCH
}

int pic_poisson(const double* rho, int32_t ncells, double dx, double V_L, double V_R, double* phi, double* E,
                void* cuda_stream) {
  PIC_ENTRY_TRY
  if (!rho || !phi || !E || ncells < 2 || ncells > PIC_MAX_CELLS_FP32 || !(dx > 0)) return PIC_EINVAL;
  PoissonParams F;
  std::memset(&F, 0, sizeof(F));
  F.rho_in = rho;
  F.mode = 2;
  F.inv_dx = 1.0 / dx;
  F.N = ncells;
  F.dx = dx;
  F.V_L = V_L;
  F.V_R = V_R;
  F.phi = phi;
  F.E = E;
  return launch_field(F, static_cast<cudaStream_t>(cuda_stream)) == cudaSuccess ? PIC_OK : PIC_ECUDA;
  PIC_ENTRY_CATCH
}

}  // extern "C"
