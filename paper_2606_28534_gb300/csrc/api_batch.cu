// api_batch.cu -- the ensemble entry points of include/pic.h (pic_batch_*).
//
// Layout.  One workspace holds, in order: the batch device words, one control block per
// simulation, the cell arrays (counts, weight sums, sort cursors, field node pairs) and node
// arrays (deposits, rho, phi, E) of all simulations back to back, the plan arrays (this much is
// zeroed by a reset), the per-simulation parameter tables of the kernels, and last the particle
// arrays: per buffer and species
// the six SoA arrays over the segments of all simulations (segment k of species s starts at a
// multiple of 1024 slots, so every TMA copy stays 16-byte aligned).
//
// Each simulation also has an ordinary pic_handle whose pointers address its segment, cells and
// nodes.  Loading, restore, snapshots, diagnostics and field output go through those handles and
// the single-simulation code; only the step itself runs the ensemble kernels:
//   k_bstep32 (persistent, every particle of every simulation) -> k_field_exact, one cluster per
//   simulation -> k_bplan (extents and work prefixes, step counter) [-> sort: scan, one cluster
//   per simulation and species, and one scatter over all tiles -> k_bplan].
// The step number lives in device memory, so a graph of 2 * sort_interval steps (two sorts: the
// buffer parity returns) is captured once per starting parity and replayed.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "api_internal.h"

using namespace picx;

struct pic_batch {
  int n = 0;
  std::vector<pic_config> cfg;
  std::vector<pic_handle*> views;
  cudaStream_t st = nullptr;   // the caller's stream
  cudaStream_t cap = nullptr;  // private stream for graph capture
  void* ws = nullptr;
  size_t ws_bytes = 0;
  bool owns_ws = false;
  size_t zero_bytes = 0;  // leading part of the workspace that starts zeroed (all but particles)
  // layout
  BatchDev* dev = nullptr;
  Ctl* ctl = nullptr;
  Species32 arr[2][2];  // [buffer][species]
  StepMaps maps[2];     // the step's stage tensor maps over arr[buffer] (both species)
  unsigned int* cnt[2] = {nullptr, nullptr};
  unsigned long long* S[2] = {nullptr, nullptr};
  unsigned int* cursor[2] = {nullptr, nullptr};
  float2* E2 = nullptr;
  long long* R[2] = {nullptr, nullptr};
  double *rho = nullptr, *phi = nullptr, *E = nullptr;
  StepParams32* d_sims[2] = {nullptr, nullptr};                  // [buffer]
  PoissonParams* d_field[2][2][2] = {};  // [buffer][sort step][step after a sort]
  SortParams* d_sort[2] = {nullptr, nullptr};                    // [source buffer]
  BSim* d_hot = nullptr;
  unsigned *pre[2] = {nullptr, nullptr}, *ncur[2] = {nullptr, nullptr};
  std::vector<unsigned long long> seg[2], cap_s[2];
  std::vector<long long> cbase, nbase;
  unsigned long long total_cap[2] = {0, 0};
  long long total_cells = 0, total_nodes = 0;
  int maxN = 0;
  // state
  int cur = 0;
  unsigned long long step = 0;
  int sort_interval = 1;
  int sms = 152;
  pic_batch_tuning tun;
  int grid_step = 0;
  cudaGraphExec_t graph[2][2] = {};  // by the buffer parity and pending scatter the graph starts from
  bool pending = false;     // a sort scan ran: the next step moves the particles to buffer 1 - cur
  int ke_every = 0;         // 1: the step sums the kinetic energy; 0: pic_batch_diag sums it
  bool ke_valid = false;    // the last step (or load) summed it
  bool prof = false;
  std::vector<EvPair> ev;
  double ms[PIC_KERNEL_KINDS] = {0};
  uint64_t launches[PIC_KERNEL_KINDS] = {0};
};

namespace {

#define CKB(x)                                \
  do {                                        \
    cudaError_t e__ = (x);                    \
    if (e__ != cudaSuccess) return PIC_ECUDA; \
  } while (0)

// Configurations that can share one batch (see include/pic.h).
bool batch_valid(const pic_config* c, int n) {
  if (!c || n < 1 || n > PIC_BATCH_MAX_SIMS || n > PIC_BATCH_MAX) return false;
  double cap[2] = {0.0, 0.0};
  for (int k = 0; k < n; ++k) {
    const pic_config& a = c[k];
    if (!valid(&a)) return false;
    if (a.precision != PIC_FP32 || a.source_mode != PIC_SOURCE_NONE || !exact_possible(a)) return false;
    if (a.neutrals || a.smooth_passes) return false;  // sheath physics: single runs only
    const pic_config& z = c[0];
    if (a.dt != z.dt || a.L / a.ncells != z.L / z.ncells || a.B != z.B || a.B_angle_deg != z.B_angle_deg ||
        a.frozen_mask != z.frozen_mask || a.field_mode != z.field_mode || a.E_ext != z.E_ext ||
        a.sort_interval != z.sort_interval)
      return false;
    for (int s = 0; s < 2; ++s) {
      if (a.mass[s] != z.mass[s] || a.charge[s] != z.charge[s]) return false;
      cap[s] += (double)capacity(&a, s);
    }
  }
  return cap[0] < 2147483648.0 && cap[1] < 2147483648.0;
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

// Segment offsets (host) and the carve of the workspace; base == nullptr only sizes it.
void layout(pic_batch* b, char* base, size_t* total) {
  const int n = b->n;
  for (int s = 0; s < 2; ++s) {
    b->seg[s].assign(n, 0);
    b->cap_s[s].assign(n, 0);
    b->total_cap[s] = 0;
  }
  b->cbase.assign(n, 0);
  b->nbase.assign(n, 0);
  b->total_cells = b->total_nodes = 0;
  b->maxN = 0;
  for (int k = 0; k < n; ++k) {
    for (int s = 0; s < 2; ++s) {
      b->cap_s[s][k] = capacity(&b->cfg[k], s);  // a multiple of 1024
      b->seg[s][k] = b->total_cap[s];
      b->total_cap[s] += b->cap_s[s][k];
    }
    b->cbase[k] = b->total_cells;
    b->nbase[k] = b->total_nodes;
    b->total_cells += b->cfg[k].ncells;
    b->total_nodes += b->cfg[k].ncells + 1;
    b->maxN = std::max(b->maxN, b->cfg[k].ncells);
  }
  Carve cv{base};
  const size_t C = (size_t)b->total_cells, M = (size_t)b->total_nodes;
  b->dev = cv.take<BatchDev>(1);
  b->ctl = cv.take<Ctl>((size_t)n);
  for (int s = 0; s < 2; ++s) {
    b->cnt[s] = cv.take<unsigned int>(C);
    b->S[s] = cv.take<unsigned long long>(C);
    b->cursor[s] = cv.take<unsigned int>(C);
  }
  b->E2 = cv.take<float2>(C);
  for (int s = 0; s < 2; ++s) b->R[s] = cv.take<long long>(M);
  b->rho = cv.take<double>(M);
  b->phi = cv.take<double>(M);
  b->E = cv.take<double>(M);
  for (int s = 0; s < 2; ++s) {
    b->pre[s] = cv.take<unsigned>((size_t)n + 1);
    b->ncur[s] = cv.take<unsigned>((size_t)n);
  }
  b->zero_bytes = (cv.off + 255) & ~size_t(255);
  // parameter tables (written once by pic_batch_init, kept by pic_batch_reset)
  for (int p = 0; p < 2; ++p) {
    b->d_sims[p] = cv.take<StepParams32>((size_t)n);
    b->d_sort[p] = cv.take<SortParams>((size_t)n);
    for (int q = 0; q < 2; ++q)
      for (int r = 0; r < 2; ++r) b->d_field[p][q][r] = cv.take<PoissonParams>((size_t)n);
  }
  b->d_hot = cv.take<BSim>((size_t)n);
  for (int p = 0; p < 2; ++p)
    for (int s = 0; s < 2; ++s) {
      Species32& a = b->arr[p][s];
      const size_t T = (size_t)b->total_cap[s];
      a.cell = cv.take<int>(T);
      a.frac = cv.take<float>(T);
      a.vx = cv.take<float>(T);
      a.vy = cv.take<float>(T);
      a.vz = cv.take<float>(T);
      a.id = cv.take<unsigned long long>(T);
    }
  *total = cv.off + 256;
}

// The single-simulation view of simulation k.
void make_view(pic_batch* b, int k, pic_handle* h) {
  h->cfg = b->cfg[k];
  h->st = b->st;
  h->N = b->cfg[k].ncells;
  h->plain = false;
  for (int s = 0; s < 2; ++s) h->cap[s] = b->cap_s[s][k];
  for (int p = 0; p < 2; ++p)
    for (int s = 0; s < 2; ++s) {
      const Species32& a = b->arr[p][s];
      const size_t o = (size_t)b->seg[s][k];
      h->a32[p][s] = Species32{a.cell + o, a.frac + o, a.vx + o, a.vy + o, a.vz + o, a.id + o};
    }
  const size_t c0 = (size_t)b->cbase[k], n0 = (size_t)b->nbase[k];
  for (int s = 0; s < 2; ++s) {
    h->cnt[s] = b->cnt[s] + c0;
    h->S[s] = b->S[s] + c0;
    h->cursor[s] = b->cursor[s] + c0;
    h->R[s] = b->R[s] + n0;
  }
  h->E2 = b->E2 + c0;
  h->rho = b->rho + n0;
  h->phi = b->phi + n0;
  h->E = b->E + n0;
  h->ctl = b->ctl + k;
  // restore staging: buffer 1 of the whole batch (restores replace every simulation)
  h->stage = reinterpret_cast<char*>(b->arr[1][0].cell);
  h->stage_bytes = (size_t)(reinterpret_cast<char*>(b->arr[1][1].id + b->total_cap[1]) - h->stage);
  derive(h);
  h->grid_step = b->sms * occupancy_step32();
  h->grid_sort = b->sms * 16;
  h->grid_diag = b->sms * 8;
}

// Kernel parameter tables of every simulation (pointers are fixed for the batch's lifetime).
int upload_tables(pic_batch* b) {
  const int n = b->n;
  std::vector<StepParams32> sims(n);
  std::vector<PoissonParams> field(n);
  std::vector<SortParams> sort(n);
  std::vector<BSim> hot(n);
  for (int p = 0; p < 2; ++p) {
    for (int k = 0; k < n; ++k) {
      pic_handle* h = b->views[k];
      const int keep_cur = h->cur;
      h->cur = p;
      sims[k] = params32(h);
      SortParams& so = sort[k];
      for (int s = 0; s < 2; ++s) {
        so.src[s] = h->a32[p][s];
        so.dst[s] = h->a32[1 - p][s];
        so.cnt[s] = h->cnt[s];
        so.cursor[s] = h->cursor[s];
        so.cap[s] = h->cap[s];
      }
      so.ctl = h->ctl;
      so.N = h->N;
      so.defer = 1;  // the scan only: the next step moves the particles
      h->cur = keep_cur;
    }
    CKB(cudaMemcpy(b->d_sims[p], sims.data(), sizeof(StepParams32) * n, cudaMemcpyHostToDevice));
    CKB(cudaMemcpy(b->d_sort[p], sort.data(), sizeof(SortParams) * n, cudaMemcpyHostToDevice));
    for (int q = 0; q < 2; ++q)
      for (int r = 0; r < 2; ++r) {
        for (int k = 0; k < n; ++k) {
          pic_handle* h = b->views[k];
          const int keep_cur = h->cur;
          h->cur = p;
          field[k] = field_params(h, q != 0, true);
          field[k].scatter_step = r;
          h->cur = keep_cur;
          if (!field[k].exact) return PIC_EINVAL;
        }
        CKB(cudaMemcpy(b->d_field[p][q][r], field.data(), sizeof(PoissonParams) * n, cudaMemcpyHostToDevice));
      }
  }
  for (int k = 0; k < n; ++k) {
    const pic_handle* h = b->views[k];
    BSim& x = hot[k];
    std::memset(&x, 0, sizeof(x));
    for (int s = 0; s < 2; ++s) {
      x.seg[s] = (unsigned)b->seg[s][k];
    }
    x.cbase = (int)b->cbase[k];
    x.N = h->N;
    x.seed = h->ph.seed;
    x.collides = h->ph.mcc_mask;
    for (int s = 0; s < 2; ++s) x.cap[s] = (unsigned)b->cap_s[s][k];
  }
  CKB(cudaMemcpy(b->d_hot, hot.data(), sizeof(BSim) * n, cudaMemcpyHostToDevice));
  return PIC_OK;
}

void bprof_begin(pic_batch* b, int kind, EvPair* e, cudaStream_t st) {
  nvtxRangePushA(kKindNames[kind]);  // a named range per launch for timeline tools (no tool: a no-op)
  e->kind = kind;
  e->a = e->b = nullptr;
  if (!b->prof) return;
  cudaEventCreate(&e->a);
  cudaEventCreate(&e->b);
  cudaEventRecord(e->a, st);
}

void bprof_end(pic_batch* b, EvPair* e, cudaStream_t st) {
  nvtxRangePop();
  if (!b->prof || !e->a) return;
  cudaEventRecord(e->b, st);
  b->ev.push_back(*e);
}

void bprof_harvest(pic_batch* b) {
  for (EvPair& e : b->ev) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, e.a, e.b) == cudaSuccess) {
      b->ms[e.kind] += ms;
      b->launches[e.kind] += 1;
    }
    cudaEventDestroy(e.a);
    cudaEventDestroy(e.b);
  }
  b->ev.clear();
}

BatchPlan plan_params(pic_batch* b, int advance) {
  BatchPlan P;
  for (int s = 0; s < 2; ++s) {
    P.pre[s] = b->pre[s];
    P.ncur[s] = b->ncur[s];
    P.sims[s] = b->d_sims[s];
  }
  P.dev = b->dev;
  P.nsims = b->n;
  P.advance = advance;
  return P;
}

// Parameters of the step kernel: in the step after a sort it reads buffer cur and fills buffer
// 1 - cur (whose per-simulation tables then serve the collision queue and births).
BatchStep32 step_params(pic_batch* b, bool scatter) {
  BatchStep32 P;
  const int dst = scatter ? 1 - b->cur : b->cur;
  for (int s = 0; s < 2; ++s) {
    P.sp[s] = b->arr[dst][s];
    P.src[s] = b->arr[b->cur][s];
    P.cursor[s] = b->cursor[s];
    P.cnt[s] = b->cnt[s];
    P.S[s] = b->S[s];
    P.pre[s] = b->pre[s];
    P.ncur[s] = b->ncur[s];
  }
  P.E2 = b->E2;
  P.ph = b->views[0]->ph;  // the shared constants (push, masses, field mode) are equal in every view
  P.sims = b->d_sims[dst];
  P.hot = b->d_hot;
  P.sum_ke = b->ke_every == 1 ? 1u : 0u;
  P.dev = b->dev;
  P.nsims = b->n;
  return P;
}

// One step of every simulation on stream st (host bookkeeping of cur and step included).
int enqueue_step(pic_batch* b, cudaStream_t st) {
  const bool sort_now = (b->step % (unsigned long long)b->sort_interval) == 0ull;
  const bool scatter = b->pending;
  EvPair e;
  bprof_begin(b, scatter ? K_STEP_SCATTER : K_STEP, &e, st);
  CKB(launch_bstep32(b->tun.variant, step_params(b, scatter), b->maps[b->cur], b->grid_step, scatter, st));
  bprof_end(b, &e, st);
  if (scatter) {
    b->cur = 1 - b->cur;
    b->pending = false;
  }
  b->ke_valid = b->ke_every == 1;
  bprof_begin(b, K_FIELD, &e, st);
  CKB(launch_field_batch(b->d_field[b->cur][sort_now ? 1 : 0][scatter ? 1 : 0], b->n, b->maxN, st));
  bprof_end(b, &e, st);
  bprof_begin(b, K_PLAN, &e, st);
  CKB(launch_bplan(plan_params(b, 1), st));
  bprof_end(b, &e, st);
  if (sort_now) {
    // the counting sort's scans: cursors now, the particles move during the next step (the extents
    // the plan just read stay those of buffer cur until then)
    bprof_begin(b, K_SORT, &e, st);
    CKB(launch_sort_scan_batch(b->d_sort[b->cur], b->n, b->maxN, st));
    bprof_end(b, &e, st);
    b->pending = true;
  }
  b->step += 1;
  return PIC_OK;
}

void drop_graphs(pic_batch* b) {
  for (int p = 0; p < 2; ++p)
    for (int q = 0; q < 2; ++q) {
      if (b->graph[p][q]) cudaGraphExecDestroy(b->graph[p][q]);
      b->graph[p][q] = nullptr;
    }
}

// Graph of 2 * sort_interval steps starting at a sort step, from buffer parity b->cur and pending
// state b->pending (both are back where they started after the two sorts).
int capture_graph(pic_batch* b) {
  const int p = b->cur;
  const bool pend = b->pending;
  const unsigned long long step0 = b->step;
  cudaGraph_t g = nullptr;
  CKB(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal));
  int rc = PIC_OK;
  for (int i = 0; i < 2 * b->sort_interval && rc == PIC_OK; ++i) rc = enqueue_step(b, b->cap);
  const cudaError_t ec = cudaStreamEndCapture(b->cap, &g);
  b->cur = p;  // capture only recorded the launches
  b->pending = pend;
  b->step = step0;
  if (rc != PIC_OK || ec != cudaSuccess || !g) {
    if (g) cudaGraphDestroy(g);
    return rc != PIC_OK ? rc : PIC_ECUDA;
  }
  cudaGraphExec_t x = nullptr;
  const cudaError_t ei = cudaGraphInstantiate(&x, g, 0);
  cudaGraphDestroy(g);
  if (ei != cudaSuccess) return PIC_ECUDA;
  b->graph[p][pend ? 1 : 0] = x;
  return PIC_OK;
}

// The plan of the current state (after init, restore or reset) and the step word.
int replan(pic_batch* b) {
  BatchDev d;
  std::memset(&d, 0, sizeof(d));
  d.step = b->step;
  CKB(cudaMemcpyAsync(b->dev, &d, sizeof(d), cudaMemcpyHostToDevice, b->st));
  CKB(launch_bplan(plan_params(b, 0), b->st));
  CKB(cudaStreamSynchronize(b->st));
  return PIC_OK;
}

// Every simulation back to its initial particles.
int load_all(pic_batch* b) {
  CKB(cudaMemsetAsync(b->ws, 0, b->zero_bytes, b->st));
  for (int k = 0; k < b->n; ++k) {
    const int rc = load_initial(b->views[k]);
    if (rc != PIC_OK) return rc;
  }
  b->cur = b->views[0]->cur;
  for (int k = 0; k < b->n; ++k)
    if (b->views[k]->cur != b->cur) return PIC_EDEVICE;
  b->step = 0;
  b->pending = false;  // the load's full sort left every simulation sorted
  b->ke_valid = true;  // and summed the kinetic energy
  return PIC_OK;
}

int sync_errors(pic_batch* b) {
  CKB(launch_bplan(plan_params(b, 0), b->st));  // gathers the simulations' error bits
  CKB(cudaStreamSynchronize(b->st));
  BatchDev d;
  CKB(cudaMemcpy(&d, b->dev, sizeof(d), cudaMemcpyDeviceToHost));
  return status_of(d.error);
}

// The view of simulation k, brought up to the batch's step and buffer (and whether the last step
// summed the kinetic energy; if not, pic_diag sums it).
pic_handle* view(pic_batch* b, int k) {
  pic_handle* h = b->views[k];
  h->step = b->step;
  h->cur = b->cur;
  h->ke_valid = b->ke_valid;
  return h;
}

}  // namespace

extern "C" {

int32_t pic_batch_variant_count(void) { return bstep32_variants(); }

const char* pic_batch_variant_name(int32_t v) { return bstep32_variant_name(v); }

int pic_batch_workspace_size(const pic_config* cfgs, int32_t nsims, size_t* bytes) {
  PIC_ENTRY_TRY
  if (!bytes || !batch_valid(cfgs, nsims)) return PIC_EINVAL;
  pic_batch tmp;
  tmp.n = nsims;
  tmp.cfg.assign(cfgs, cfgs + nsims);
  layout(&tmp, nullptr, bytes);
  return PIC_OK;
  PIC_ENTRY_CATCH
}

int pic_batch_init(const pic_config* cfgs, int32_t nsims, void* workspace, size_t workspace_bytes,
                   void* cuda_stream, pic_batch** out) {
  PIC_ENTRY_TRY
  if (!out) return PIC_EINVAL;
  *out = nullptr;
  if (!batch_valid(cfgs, nsims)) return PIC_EINVAL;
  if (workspace && (reinterpret_cast<uintptr_t>(workspace) & 255u)) return PIC_EINVAL;
  pic_batch* b = new (std::nothrow) pic_batch();
  if (!b) return PIC_ENOMEM;
  try {
    b->n = nsims;
    b->cfg.assign(cfgs, cfgs + nsims);
    b->st = static_cast<cudaStream_t>(cuda_stream);
    b->sort_interval = cfgs[0].sort_interval;
    size_t need = 0;
    layout(b, nullptr, &need);
    if (workspace) {
      if (workspace_bytes < need) {
        delete b;
        return PIC_ENOMEM;
      }
      b->ws = workspace;
    } else {
      if (cudaMalloc(&b->ws, need) != cudaSuccess) {
        delete b;
        return PIC_ENOMEM;
      }
      b->owns_ws = true;
    }
    b->ws_bytes = need;
    layout(b, static_cast<char*>(b->ws), &need);
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, dev);
    if (b->sms <= 0) b->sms = 152;
    *out = b;
    int rc = PIC_OK;
    if (cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking) != cudaSuccess) rc = PIC_ECUDA;
    b->views.assign(nsims, nullptr);
    for (int k = 0; k < nsims && rc == PIC_OK; ++k) {
      b->views[k] = new (std::nothrow) pic_handle();
      if (!b->views[k]) {
        rc = PIC_ENOMEM;
        break;
      }
      make_view(b, k, b->views[k]);
      if (make_step_maps(b->views[k]) != PIC_OK) rc = PIC_ECUDA;  // the single-run steps of a view
    }
    for (int p = 0; p < 2 && rc == PIC_OK; ++p)
      if (encode_step_maps(b->arr[p], b->total_cap, &b->maps[p]) != PIC_OK) rc = PIC_ECUDA;
    if (rc == PIC_OK) {
      pic_batch_tuning t;
      std::memset(&t, 0, sizeof(t));
      t.use_graph = 1;
      rc = pic_batch_set_tuning(b, &t);
    }
    if (rc == PIC_OK) rc = load_all(b);
    if (rc == PIC_OK) rc = upload_tables(b);
    if (rc == PIC_OK) rc = replan(b);
    if (rc == PIC_OK) rc = sync_errors(b);
    if (rc != PIC_OK) {
      pic_batch_free(b);
      *out = nullptr;
    }
    return rc;
  } catch (...) {  // a host allocation or thread failed part way: release what was taken
    pic_batch_free(b);
    *out = nullptr;
    return PIC_ENOMEM;
  }
  PIC_ENTRY_CATCH
}

int pic_batch_set_tuning(pic_batch* b, const pic_batch_tuning* t) {
  PIC_ENTRY_TRY
  if (!b || !t) return PIC_EINVAL;
  if (t->variant < 0 || t->variant >= bstep32_variants()) return PIC_EINVAL;
  const int occ = bstep32_occupancy(t->variant);
  if (t->ctas_per_sm < 0 || t->ctas_per_sm > occ) return PIC_EINVAL;
  if (b->cap) cudaStreamSynchronize(b->st);
  drop_graphs(b);
  b->tun = *t;
  b->grid_step = b->sms * (t->ctas_per_sm ? t->ctas_per_sm : occ);
  return PIC_OK;
  PIC_ENTRY_CATCH
}

int pic_batch_set_diag_interval(pic_batch* b, int32_t every) {
  PIC_ENTRY_TRY
  if (!b || every < 0 || every > 1) return PIC_EINVAL;
  if (every != b->ke_every) {
    cudaStreamSynchronize(b->st);
    drop_graphs(b);  // the graphs hold the kernel parameters of the other choice
  }
  b->ke_every = every;
  return PIC_OK;
  PIC_ENTRY_CATCH
}

int pic_batch_get_tuning(pic_batch* b, pic_batch_tuning* t) {
  PIC_ENTRY_TRY
  if (!b || !t) return PIC_EINVAL;
  *t = b->tun;
  return PIC_OK;
  PIC_ENTRY_CATCH
}

int pic_batch_step(pic_batch* b, int32_t n) {
  PIC_ENTRY_TRY
  if (!b || n < 0) return PIC_EINVAL;
  const unsigned long long cycle = 2ull * (unsigned long long)b->sort_interval;
  while (n > 0) {
    const bool graphable = b->tun.use_graph && !b->prof && (b->step % (unsigned long long)b->sort_interval) == 0ull &&
                           (unsigned long long)n >= cycle;
    if (graphable) {
      cudaGraphExec_t& g = b->graph[b->cur][b->pending ? 1 : 0];
      if (!g) {
        const int rc = capture_graph(b);
        if (rc != PIC_OK) return rc;
      }
      CKB(cudaGraphLaunch(g, b->st));
      b->step += cycle;  // two sorts: the buffer parity and the pending state are back where they started
      b->ke_valid = b->ke_every == 1;
      n -= (int32_t)cycle;
    } else {
      const int rc = enqueue_step(b, b->st);
      if (rc != PIC_OK) return rc;
      n -= 1;
    }
  }
  return PIC_OK;
  PIC_ENTRY_CATCH
}

int pic_batch_sync(pic_batch* b) {
  PIC_ENTRY_TRY
  if (!b) return PIC_EINVAL;
  return sync_errors(b);
  PIC_ENTRY_CATCH
}

int pic_batch_diag(pic_batch* b, pic_diag_t* out, int32_t nsims) {
  PIC_ENTRY_TRY
  if (!b || !out || nsims < 0 || nsims > b->n) return PIC_EINVAL;
  for (int k = 0; k < nsims; ++k) {
    const int rc = pic_diag(view(b, k), out + k);
    if (rc != PIC_OK) return rc;
  }
  return PIC_OK;
  PIC_ENTRY_CATCH
}

int pic_batch_snapshot(pic_batch* b, int32_t k, void* buf, size_t cap, size_t* needed) {
  PIC_ENTRY_TRY
  if (!b || k < 0 || k >= b->n) return PIC_EINVAL;
  return pic_snapshot(view(b, k), buf, cap, needed);
  PIC_ENTRY_CATCH
}

int pic_batch_restore(pic_batch* b, const void* const* blobs, const size_t* lens) {
  PIC_ENTRY_TRY
  if (!b || !blobs || !lens) return PIC_EINVAL;
  unsigned long long step = 0;
  for (int k = 0; k < b->n; ++k) {
    unsigned long long sk = 0;
    if (!blob_step(blobs[k], lens[k], &sk)) return PIC_ECORRUPT;
    if (k == 0) step = sk;
    if (sk != step) return PIC_EINVAL;
  }
  // every blob is checked before any state changes
  for (int k = 0; k < b->n; ++k) {
    const int rc = check_blob(b->views[k], blobs[k], lens[k]);
    if (rc != PIC_OK) return rc;
  }
  CKB(cudaStreamSynchronize(b->st));
  for (int k = 0; k < b->n; ++k) {
    const int rc = restore_state(b->views[k], blobs[k], lens[k], true);
    if (rc != PIC_OK) return rc;
  }
  for (int k = 0; k < b->n; ++k) {
    pic_handle* h = b->views[k];
    int rc = refresh_field(h);
    if (rc == PIC_OK) rc = check_errors(h);
    if (rc != PIC_OK) return rc;
  }
  b->cur = b->views[0]->cur;
  b->step = step;
  b->pending = false;
  b->ke_valid = true;
  const int rc = replan(b);
  if (rc != PIC_OK) return rc;
  return sync_errors(b);
  PIC_ENTRY_CATCH
}

int pic_batch_reset(pic_batch* b) {
  PIC_ENTRY_TRY
  if (!b) return PIC_EINVAL;
  CKB(cudaStreamSynchronize(b->st));
  int rc = load_all(b);
  if (rc == PIC_OK) rc = replan(b);
  if (rc == PIC_OK) rc = sync_errors(b);
  return rc;
  PIC_ENTRY_CATCH
}

int pic_batch_get_field(pic_batch* b, int32_t k, int64_t* R, double* rho, double* phi, float* E, size_t nnodes) {
  PIC_ENTRY_TRY
  if (!b || k < 0 || k >= b->n) return PIC_EINVAL;
  return pic_get_field(view(b, k), R, rho, phi, E, nnodes);
  PIC_ENTRY_CATCH
}

int pic_batch_storage_order(pic_batch* b, int32_t k, int32_t species, int32_t* cell, uint64_t* ids, size_t cap,
                            size_t* n) {
  PIC_ENTRY_TRY
  if (!b || k < 0 || k >= b->n) return PIC_EINVAL;
  return pic_storage_order(view(b, k), species, cell, ids, cap, n);
  PIC_ENTRY_CATCH
}

int pic_batch_profile(pic_batch* b, int enable) {
  PIC_ENTRY_TRY
  if (!b) return PIC_EINVAL;
  if (!enable && b->prof) {
    cudaStreamSynchronize(b->st);
    bprof_harvest(b);
  }
  b->prof = enable != 0;
  return PIC_OK;
  PIC_ENTRY_CATCH
}

int pic_batch_kernel_times(pic_batch* b, double* ms, uint64_t* launches, const char** names, int32_t nkinds) {
  PIC_ENTRY_TRY
  if (!b || nkinds < 0) return PIC_EINVAL;
  CKB(cudaStreamSynchronize(b->st));
  bprof_harvest(b);
  for (int k = 0; k < nkinds && k < PIC_KERNEL_KINDS; ++k) {
    if (ms) ms[k] = b->ms[k];
    if (launches) launches[k] = b->launches[k];
    if (names) names[k] = kKindNames[k];
  }
  for (int k = 0; k < PIC_KERNEL_KINDS; ++k) {
    b->ms[k] = 0.0;
    b->launches[k] = 0;
  }
  return PIC_OK;
  PIC_ENTRY_CATCH
}

void pic_batch_free(pic_batch* b) {
  if (!b) return;
  cudaStreamSynchronize(b->st);
  bprof_harvest(b);
  drop_graphs(b);
  for (pic_handle* h : b->views) delete h;
  if (b->cap) cudaStreamDestroy(b->cap);
  if (b->owns_ws && b->ws) cudaFree(b->ws);
  delete b;
}

}  // extern "C"
