// api_internal.h -- host-side state of a simulation handle and the helpers of api.cu that the
// ensemble entry points (api_batch.cu) share: an ensemble keeps one handle per simulation whose
// pointers address that simulation's part of the ensemble's arrays.
#pragma once
#include <vector>

// Entry points catch what their host code may throw (a host allocation that fails, a host thread
// that cannot start), so that no C++ exception crosses the C ABI: the call returns PIC_ENOMEM.
#define PIC_ENTRY_TRY try {
#define PIC_ENTRY_CATCH \
  }                     \
  catch (...) {         \
    return PIC_ENOMEM;  \
  }

#include "../../include/pic.h"
#include "pic_internal.cuh"

int occupancy_step32(bool scatter = false);
int occupancy_step64();

namespace picx {

enum Kind { K_STEP = 0, K_SOURCE, K_FIELD, K_SORT, K_LOAD, K_DIAG, K_PLAN, K_STEP_SCATTER, K_NEUTRAL, K_NEUTRAL_COMPACT, K_KINDS };
extern const char* const kKindNames[PIC_KERNEL_KINDS];

struct EvPair {
  int kind;
  cudaEvent_t a, b;
};

}  // namespace picx

struct pic_handle {
  pic_config cfg;
  cudaStream_t st = nullptr;
  void* ws = nullptr;
  size_t ws_bytes = 0;
  bool owns_ws = false;
  int N = 0;
  bool plain = false;
  unsigned long long cap[2] = {0, 0};
  Species32 a32[2][2];  // [buffer][species]
  int cur = 0;
  Species64 a64[2];
  StepMaps maps[2];             // the particle step's stage tensor maps, per buffer (FP32 path)
  bool maps_ok = false;         // maps made (make_step_maps): particle steps may be launched
  FieldGrid* fgrid = nullptr;  // scratch of the grid-wide field solve (FP32 path)
  int field_ctas = 0;          // its CTAs (0: the one-cluster solve)
  unsigned int* cnt[2] = {nullptr, nullptr};
  unsigned long long* S[2] = {nullptr, nullptr};
  unsigned int* cursor[2] = {nullptr, nullptr};
  double* acc[2] = {nullptr, nullptr};
  long long* R[2] = {nullptr, nullptr};
  double *rho = nullptr, *phi = nullptr, *E = nullptr;
  float2* E2 = nullptr;
  Ctl* ctl = nullptr;
  char* stage = nullptr;  // FP32 restore: device staging for a blob's arrays (unused between sorts)
  size_t stage_bytes = 0;
  Phys ph;
  unsigned long long step = 0;
  int grid_step = 0, grid_sort = 0, grid_diag = 0, grid_scatter = 0;
  int ke_every = 0;       // the step sums the kinetic energy on every ke_every-th step (0: never)
  bool pending_scatter = false;  // a sort scan ran: the next step moves the particles to buffer 1 - cur
  bool open_sort = false, open_scatter = false;  // the step in progress sorts / moved the particles
  bool split_open = false;  // pic_step_begin ran; pic_step_end closes the step
  bool ke_valid = false;  // the last completed step (or refresh) summed it (ke_last holds it)
  // tracked neutrals (cfg.neutrals): two compacted buffers, the one the next step reads is nt_buf
  unsigned long long cap_nt = 0;
  Species32 nt[2];
  int nt_buf = 0;
  float2* NE2 = nullptr;       // node electron density pairs per cell
  unsigned int* wlog = nullptr;  // ions absorbed at a wall in the current step (recycling)
  int grid_neutral = 0;
  bool prof = false;
  std::vector<picx::EvPair> ev;
  std::vector<cudaEvent_t> ev_free;  // harvested events, reused (creating one costs host time)
  double ms[PIC_KERNEL_KINDS] = {0};
  uint64_t launches[PIC_KERNEL_KINDS] = {0};
};

namespace picx {

bool valid(const pic_config* c);
unsigned long long capacity(const pic_config* c, int s);
unsigned long long neutral_capacity(const pic_config* c);
void derive(pic_handle* h);
void prof_begin(pic_handle* h, int kind, EvPair* e);
void prof_end(pic_handle* h, EvPair* e);
void prof_harvest(pic_handle* h);
StepParams32 params32(pic_handle* h);
bool exact_possible(const pic_config& c);
PoissonParams field_params(pic_handle* h, bool keep_counts, bool count_step);
int refresh_field(pic_handle* h);
int check_errors(pic_handle* h);
// The two halves of pic_step's step: the particle phase, and the field solve (of R_total when not
// null), bookkeeping and sort scan that close it.
int step_particles(pic_handle* h);
int step_close(pic_handle* h, const long long* R_total);
int status_of(unsigned int err_bits);
// Initial particles of h (the grid arrays and the control block are already zero): load,
// padding, control block, deposit + field + sort, error check.
int load_initial(pic_handle* h);
// Every check pic_restore makes of a blob before it changes any state: format, checksum,
// configuration hash, sizes, capacity, the range of every cell and fraction.
int check_blob(const pic_handle* h, const void* buf, size_t len);
// The particle step's stage tensor maps of a handle (api.cu); PIC_ECUDA if they cannot be made.
int make_step_maps(pic_handle* h);
// The same for species arrays a[2] of capacities cap[2] (an ensemble's batch-wide arrays).
int encode_step_maps(const Species32* a, const unsigned long long* cap, StepMaps* out);
// Everything pic_restore does before the redeposit: (unless checked) check_blob, particles into
// buffer 0 (FP32: through h->stage), control block, cleared accumulators, h->step.  Leaves
// h->cur = 0.
int restore_state(pic_handle* h, const void* buf, size_t len, bool checked);
// Step number recorded in a snapshot blob (no other check).
bool blob_step(const void* buf, size_t len, unsigned long long* step);

}  // namespace picx
