// pic_internal.cuh -- device-side data layout and helpers of the GB300 PIC MC library.
//
// Layout in HBM (one handle):
//   per species s, two particle buffers (A/B, swapped by the counting sort), SoA:
//     cell int32[cap] | frac f32[cap] | vx f32[cap] | vy f32[cap] | vz f32[cap] | id u64[cap]
//   (PIC_FP64_PLAIN: one buffer, x f64[cap] (cell units) | vx, vy, vz f64[cap] | id u64[cap])
//   grid: cnt_s u32[N], S_s u64[N] (per-cell particle count and sum of right CIC weights),
//         R_s i64[N+1], rho f64[N+1], phi f64[N+1], E f64[N+1], E2 float2[N] = (E_c, E_{c+1}),
//         cursor_s u32[N] (sort), plain path rho_acc_s f64[N+1]
//   control block Ctl (counters and array extents), 256-byte aligned.
// Extents n_cur are kept a multiple of 4 so that every particle load/store is a 128-bit access;
// slots past the last particle carry cell = DEAD_CELL.
// The cell word of a live particle is cell | k << 18 | c << 30: the cell (N < 2^18) and the
// particle's null-collision countdown (k, c) (the geometric countdown reading; k in 1..4095, c set
// when its expiry is a candidate; both 0 for species without the test).  DEAD_CELL has bit 31 set,
// which no live word has.  The plain FP64 path keeps the pair (k | c << 12) in its own array.
#pragma once
#include <cuda.h>  // CUtensorMap (the descriptor type only; no driver call is linked)
#include <cuda_runtime.h>
#include <stdint.h>

#ifndef PIC_TPB
#define PIC_TPB 256  // threads per CTA of the particle kernels
#endif
#define PIC_PPT 4  // particles per thread (one 128-bit access per array)
#ifndef PIC_STEP_MINB
#define PIC_STEP_MINB 3  // resident CTAs per SM the step kernel is compiled for
#endif
#define PIC_TILE (PIC_TPB * PIC_PPT)
#define PIC_WCAP 2048
#define PIC_DEAD_CELL ((int)0x80000000)
#define PIC_CELL_BITS 18
#define PIC_CELL_MASK ((1 << PIC_CELL_BITS) - 1)
#define PIC_NEXT_KMAX 4095u       // largest countdown
#define PIC_NEXT_CAND (1u << 12)  // in a countdown pair k | c << 12: the expiry is a candidate
#define PIC_FIELD_CTAS 8
#define PIC_FIELD_TPB 1024
#define PIC_FIELD_SEG_MAX 24576  // nodes per CTA of the field cluster (192 KB of shared memory)
#define PIC_MAX_CELLS_FP32 (PIC_FIELD_CTAS * PIC_FIELD_SEG_MAX - 1)

// Philox counter word 2: the stream of a draw
#define CH_INIT 1u
#define CH_COLL 2u
#define CH_SCAT 3u
#define CH_CHILD 4u
#define CH_SOURCE 5u
#define CH_RECYCLE 6u
#define CH_NIZ 7u
#define PIC_MAX_SMOOTH 4

// error bits of Ctl::error
#define ERR_OVERFLOW 1u
#define ERR_TIMEOUT 2u
#define ERR_DEVICE 4u

#define PIC_DIAG_BLOCKS 64  // node blocks of the field-energy reduction (fixed: reproducible sums)

struct Ctl {
  unsigned long long n_cur[2];   // array extent (multiple of 4, includes dead slots)
  unsigned long long n_born[2];  // slots claimed past n_cur in the current step
  unsigned long long n_live[2];  // live particles
  unsigned long long wall_hits[2][2];
  unsigned long long coll[5];
  unsigned long long near_thr[2];
  unsigned long long viol[2];
  unsigned long long births[2];
  unsigned long long source_pairs;
  unsigned long long dropped;
  long long wall_charge;
  unsigned long long wall_energy_fx[2];  // sum of 0.5 m v^2 of absorbed particles, 2^-24 units
  unsigned long long src_K;              // ions absorbed in the current step
  unsigned long long sort_total[2];
  unsigned long long sort_new[2];        // deferred sort: extent of the buffer the next step fills
  unsigned int sort_done;                // blocks of the scatter that finished
  unsigned int error;
  unsigned long long ke_fx[2];           // diag scratch: sum 0.5 m v^2, 2^-24 units
  unsigned long long particle_steps;     // sum over steps of the live particles at step start
  unsigned long long live_mark;          // live particles at the start of the next step
  unsigned long long ke_acc[2];          // sum of ke_fx32 over the particles alive after this step
  unsigned long long ke_last[2];         // ke_acc of the last completed step (read by pic_diag)
  long long netq;                        // diag scratch: sum_j sum_s sign(q_s) R_sj
  double fe_part[PIC_DIAG_BLOCKS];       // diag scratch: field energy per block of nodes
  // tracked neutrals (species 2)
  unsigned long long nt_cur;             // extent of the neutral buffer read by the next step
  unsigned long long nt_out;             // neutrals written by the current step (next extent)
  unsigned long long nt_live;
  unsigned long long nt_recycled[2], nt_lost[2], nt_ionized, nt_near, nt_particle_steps;
  unsigned long long nt_ke_fx;           // diag scratch: sum 0.5 m v^2 of the neutrals, 2^-24 units
  unsigned long long wlog_n;             // ions absorbed at a wall in the current step (recycling log)
  unsigned long long diag_step;          // steps taken when the last diagnostics were enqueued
  unsigned long long diag_what;          // PIC_DIAG_* of that request
  // the ordinary particle step's chunk schedule: chunks claimed per species, CTAs done (the last
  // CTA of a launch zeroes all three for the next launch)
  unsigned int chunk_claim[2];
  unsigned int chunk_done;
  unsigned int chunk_pad;
};

struct Species32 {
  int* cell;
  float* frac;
  float* vx;
  float* vy;
  float* vz;
  unsigned long long* id;
};

struct Species64 {
  double* x;
  double* vx;
  double* vy;
  double* vz;
  unsigned long long* id;
  unsigned* nk;  // null-collision countdown pair k | c << 12 (0: no test)
};

// Physics constants of one species, rounded once on the host.
struct SpConst {
  float qmdt2;      // (q/m) dt / 2
  float t[3], s[3]; // Boris rotation vectors
  float p_null;     // 1 - exp(-nu_max dt), FP32
  unsigned p_null_u24;  // ceil(p_null 2^24): (w >> 8) < p_null_u24  <=>  u01(w) < p_null
  float lnq;        // log1p(-p_null) rounded to FP32 (the countdown's fast path)
  double lnq_d;     // log1p(-p_null) in FP64
  float nu_max;     // FP32
  float mass;
  float vt;         // sqrt(T/m) (source, load)
  float w;          // weight dx/ppc
  int qsign;        // sign of the charge
  double qmdt2_d, t_d[3], s_d[3], mass_d, vt_d;
};

struct Phys {
  SpConst sp[2];
  float dtdx;
  float ngs_el, ngs_ex, ngs_iz, ngs_cx;  // n_gas * sigma
  float E_ex, E_iz, inv_E_ex, inv_E_iz;
  float two_m_over_M;
  float vt_gas;  // sqrt(Tg / m_ion)
  float E_ext;
  float src_x1;
  double dtdx_d, ngs_el_d, ngs_ex_d, ngs_iz_d, ngs_cx_d, E_ex_d, E_iz_d, two_m_over_M_d,
      vt_gas_d, E_ext_d, src_x1_d;
  unsigned int coll_mask, field_mode, push_mask, has_B;
  unsigned int mcc_mask;  // bit s: species s takes the null-collision test (processes on, pushed, p_null > 0)
  int N;
  unsigned long long seed;
};

struct StepParams32 {
  Species32 sp[2];
  unsigned long long cap[2];
  const float2* E2;
  unsigned int* cnt[2];
  unsigned long long* S[2];
  Ctl* ctl;
  Phys ph;
  unsigned long long step;
  unsigned int sum_ke;   // sum the kinetic energy of the particles alive after this step
  unsigned int scatter;  // the step after a sort: read src, write each particle to its sorted slot in sp
  Species32 src[2];      // scatter: the buffer the sort step left (sp: the buffer being filled)
  unsigned int* cursor[2];  // scatter: per-cell write cursors of the sort scan
  unsigned int* wlog;    // recycling: index of each ion absorbed at a wall in the buffer the step
                         // reads, | side << 31 (null: no recycling)
};

// The particle step's stage loads (a kernel parameter of its own): per species, a 2-D tensor map
// over the five 4-byte arrays of the buffer the step reads (rows cell, frac, vx, vy, vz, each
// cap[s] elements apart), so that a chunk's stage is one tensor copy of a 128 x 5 box.
struct StepMaps {
  CUtensorMap tmap[2];
};

// The neutral step (k_neutral.cu): the neutrals alive at the step start move, leave at the walls
// or ionize; the ions the particle step logged at the walls return as neutrals.  In place (dst ==
// src, new neutrals appended), or compacted into the other buffer on the steps that sort.
struct NeutralParams {
  StepParams32 P;                   // the particle step's parameters (births, deposits, counters)
  Species32 src, dst;               // neutral buffers read / written
  unsigned long long cap;           // neutral capacity
  const unsigned long long* ion_id; // ion ids of the buffer the particle step read (log indices)
  const float2* NE2;                // node electron density pairs (n_e,c, n_e,c+1) per cell
  float Kdt;                        // K_iz dt
  float vt_rec, vt_sec;             // sqrt(T_rec / m_ion), sqrt(T_sec / m_e)
  float mass;                       // neutral (= ion) mass
  unsigned recycle_u24;             // ceil(recycle 2^24): (w >> 8) < recycle_u24  <=>  u01(w) < recycle
  int ionize;                       // K_iz > 0
};

struct StepParams64 {
  Species64 sp[2];
  unsigned long long cap[2];
  const double* E;
  double* acc[2];  // rho accumulators (particle units) at N + 1 nodes
  Ctl* ctl;
  Phys ph;
  unsigned long long step;
};

// --------------------------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds; each round forms the two
// 32x32 -> 64-bit products of counter words 0 and 2 with the round multipliers and mixes their
// halves with words 1, 3 and the key; the key advances by the two Weyl increments between rounds.
// The high and low halves are separate 32-bit multiplies: a caller that uses only some output
// words (the null-collision test reads word 0) lets the compiler drop the products of the last
// two rounds that feed nothing (measured: 2.7% off the particle step against 64-bit products).
__device__ __forceinline__ uint4 philox10(uint4 c, uint2 k) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const unsigned h0 = __umulhi(0xD2511F53u, c.x), l0 = 0xD2511F53u * c.x;
    const unsigned h1 = __umulhi(0xCD9E8D57u, c.z), l1 = 0xCD9E8D57u * c.z;
    c = make_uint4(h1 ^ c.y ^ k.x, l1, h0 ^ c.w ^ k.y, l0);
    k.x += 0x9E3779B9u;
    k.y += 0xBB67AE85u;
  }
  return c;
}

// The draw for (particle id, step, channel, index): key (step lo, seed lo) -- the same for every
// particle of a step, so the key schedule is warp-uniform -- and counter (id lo, id hi,
// channel | step hi << 8, index ^ seed hi).
__device__ __forceinline__ uint4 draw4(unsigned long long id, unsigned long long seed,
                                       unsigned long long step, unsigned ch, unsigned idx) {
  return philox10(make_uint4((unsigned)id, (unsigned)(id >> 32), ch | ((unsigned)(step >> 32) << 8),
                             idx ^ (unsigned)(seed >> 32)),
                  make_uint2((unsigned)step, (unsigned)seed));
}

// Checked builds (-DPIC_CHECKED, build.py's checked library): a particle whose stored cell is
// neither a cell of the grid nor the dead mark is reported (ERR_DEVICE) and treated as dead instead
// of being used as an index.  Ordinary builds compile the test away.
#ifdef PIC_CHECKED
#define PIC_CHECKED_BUILD 1
#else
#define PIC_CHECKED_BUILD 0
#endif
__device__ __forceinline__ int checked_cell(int c, int N, unsigned int* error) {
  if (PIC_CHECKED_BUILD && c != PIC_DEAD_CELL && (c < 0 || (c & PIC_CELL_MASK) >= N)) {
    atomicOr(error, ERR_DEVICE);
    return PIC_DEAD_CELL;
  }
  return c;
}

// 24-bit uniform in [0, 1): exact in FP32 and FP64
__device__ __forceinline__ float u01f(unsigned w) { return (float)(w >> 8) * 5.9604644775390625e-08f; }
__device__ __forceinline__ double u01d(unsigned w) { return (double)(w >> 8) * 5.9604644775390625e-08; }

// The countdown pair G(w) (k | c << 12) from one Philox word w: u = (w >> 8) 2^-24,
// r = log(1 - u) / log1p(-p_null), K = 1 + floor(r); (K, candidate) if K <= 4095, else (4095, not a
// candidate: the particle waits 4095 steps and draws again).  The FP32 quotient (logf and the
// division within 1 ulp and 0.5 ulp, log1p(-p_null) rounded once: relative error below 2.5e-7)
// decides the floor unless it lies within 1e-6 r (at least 1e-6) of an integer; then the quotient is
// taken in FP64 (log within 1 ulp).  A draw whose FP64 quotient lies within 1e-9 max(1, r) of an
// integer is counted as near-threshold.
__device__ __forceinline__ unsigned countdown_draw(const SpConst& K, unsigned w, unsigned* near) {
  const float v = 1.0f - u01f(w);  // (0, 1], exact
  const float r = logf(v) / K.lnq;
  float fl = floorf(r);
  if (!(fminf(r - fl, fl + 1.0f - r) > 1e-6f * fmaxf(r, 1.0f))) {
    const double rd = log((double)v) / K.lnq_d;
    const double fd = floor(rd);
    const double tol = 1e-9 * fmax(1.0, rd);
    if (near && rd > 0.0 && (rd - fd < tol || fd + 1.0 - rd < tol)) atomicAdd(near, 1u);
    if (fd >= (double)PIC_NEXT_KMAX) return PIC_NEXT_KMAX;
    return ((unsigned)fd + 1u) | PIC_NEXT_CAND;
  }
  if (fl >= (float)PIC_NEXT_KMAX) return PIC_NEXT_KMAX;
  return ((unsigned)fl + 1u) | PIC_NEXT_CAND;
}

// The same pair with the quotient in FP64 throughout (the plain FP64 path).
__device__ __forceinline__ unsigned countdown_draw_d(const SpConst& K, unsigned w, unsigned* near) {
  const double rd = log(1.0 - u01d(w)) / K.lnq_d;
  const double fd = floor(rd);
  const double tol = 1e-9 * fmax(1.0, rd);
  if (near && rd > 0.0 && (rd - fd < tol || fd + 1.0 - rd < tol)) atomicAdd(near, 1u);
  if (fd >= (double)PIC_NEXT_KMAX) return PIC_NEXT_KMAX;
  return ((unsigned)fd + 1u) | PIC_NEXT_CAND;
}

// The countdown pair of a particle of species s created in step `step` (the load: step 0; births,
// source pairs, the products of a neutral's ionization): from word 0 of Philox(id, step, INIT, 2);
// 0 for a species without the null-collision test.
template <bool FP64 = false>
__device__ __forceinline__ unsigned created_pair(const Phys& ph, int s, unsigned long long id,
                                                 unsigned long long step) {
  if (!((ph.mcc_mask >> s) & 1u)) return 0u;
  const uint4 w = draw4(id, ph.seed, step, CH_INIT, 2u);
  return FP64 ? countdown_draw_d(ph.sp[s], w.x, nullptr) : countdown_draw(ph.sp[s], w.x, nullptr);
}

// The cell word of such a particle in cell c.
__device__ __forceinline__ int created_word(const Phys& ph, int s, int c, unsigned long long id,
                                            unsigned long long step) {
  return c | (int)(created_pair(ph, s, id, step) << PIC_CELL_BITS);
}


__host__ __device__ inline unsigned long long round_up4(unsigned long long n) { return (n + 3ull) & ~3ull; }

// Kinetic energy of one FP32 particle in 2^-24 fixed point with every rounding spelled out (no
// contraction), so the sum over particles is exact and independent of order and of the kernel
// that forms it: rint(2^24 * (m/2) * ((vx^2 + vy^2) + vz^2)), all products and sums in FP32.
__device__ __forceinline__ unsigned long long ke_fx32(float vx, float vy, float vz, float mass) {
  const float t = __fadd_rn(__fadd_rn(__fmul_rn(vx, vx), __fmul_rn(vy, vy)), __fmul_rn(vz, vz));
  return __float2ull_rn(__fmul_rn(__fmul_rn(__fmul_rn(0.5f, mass), t), 16777216.0f));
}

// --------------------------------------------------------------------------------------------
// Bulk asynchronous copies (TMA, 1D) and mbarriers, inline PTX for sm_90+.
__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_init_fence() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0u;
}
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
#define PIC_WAIT_LIMIT_NS 1000000000ull  // a bounded wait gives up after about one second
// Wait for a phase for at most PIC_WAIT_LIMIT_NS of wall time (and at most 2^22 polls); false when
// the limit ran out (the caller reports it).  The first poll usually succeeds and costs no timer read.
__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long* bar, unsigned parity) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = global_ns();
  for (int it = 1; it < (1 << 22); ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((it & 63) == 0 && global_ns() - t0 > PIC_WAIT_LIMIT_NS) return false;
  }
  return false;
}
// Order this thread's earlier generic-proxy accesses of shared memory before later async-proxy
// (TMA) accesses, so that a stage buffer is refilled only after it has been read.
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
// Global -> shared tiled tensor copy of the box at (x, y) of a 2-D tensor map (in kernel parameter
// space); completes the box's bytes on the mbarrier.  x times the element size a multiple of 16.
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::
          "r"(smem_u32(dst)),
      "l"(reinterpret_cast<unsigned long long>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}
// Global -> shared bulk copy; completes tx bytes on the mbarrier.  Both addresses 16-byte aligned,
// size a multiple of 16.
__device__ __forceinline__ void tma_load_1d(void* dst, const void* src, unsigned bytes, unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// launchers (each file owns its kernels)
// Scratch of the grid-wide integer-exact field solve of one simulation (k_field_grid): the
// arrival count and generation of its grid barrier, and the per-CTA totals it exchanges
// (interior charge, first moment).  Zero-initialised with the workspace.
constexpr int PIC_FIELD_GRID_MAX = 1024;  // CTAs of the grid-wide solve
struct FieldGrid {
  unsigned int count;
  unsigned int gen;
  unsigned int pad[2];
  __int128 tot[PIC_FIELD_GRID_MAX][2];
};

struct PoissonParams {
  // input: either fixed-point counts (cnt/S) or FP64 accumulators (acc) or a plain rho
  const unsigned int* cnt[2];
  unsigned long long* S[2];
  double* acc[2];
  const double* rho_in;
  double qw[2];     // q_s * w_s
  long long m[2];   // exact path: integer charge multipliers q_s ppc_{1-s} / gcd(ppc_0, ppc_1)
  double e_in, e_wall, e_bias;  // exact path: E coefficients (see k_field.cu)
  double inv_dx;
  int exact;        // mode 0: integer-exact field (integer charges)
  int mode;         // 0: fixed point, 1: FP64 accumulators, 2: plain rho, 3: from stored R
  int zero_R;       // mode 3: R is zeroed once read (the adjoint forward's next deposit)
  int keep_counts;  // fixed point: leave cnt for the sort
  int N;
  double dx, V_L, V_R;
  long long* R[2];  // out (fixed point mode)
  double* rho;      // out (modes 0, 1)
  double* phi;
  double* E;
  float2* E2;       // out, may be null
  Ctl* ctl;         // bookkeeping, may be null
  int count_step;   // add the live particles at the start of this step to particle_steps
  Species32 pad32[2];
  Species64 pad64[2];
  unsigned long long cap[2];
  int plain;
  int scatter_step;  // bookkeeping after a scattering step: the extent of the filled buffer is sort_new
  int smooth;        // density smoothing passes (exact path and mode 3)
  float2* NE2;       // out, may be null: node electron density pairs per cell (neutral ionization)
  double ne_scale;   // n_e,j = R_0j ne_scale (x 2 at the wall nodes)
  Species32 nt_pad;  // neutrals: the buffer the neutral step wrote (padded to a multiple of 4)
  unsigned long long nt_cap;  // 0: no neutrals
  int nt_append;     // the neutral step ran in place: its new neutrals follow the old extent
  const long long* R_in;  // exact path: the node deposits to solve (2 (N+1): species 0, then 1) in
                          // place of this handle's own counts (a decomposed simulation's total)
  int no_book;       // skip the per-step bookkeeping (a re-solve outside a step)
  FieldGrid* grid;   // exact path: solve over grid_ctas co-resident CTAs (null: one cluster)
  int grid_ctas;
};

struct SortParams {
  Species32 src[2], dst[2];
  unsigned int* cnt[2];
  unsigned int* cursor[2];
  unsigned long long cap[2];
  Ctl* ctl;
  int N;
  int defer;  // 1: record the new extent in sort_new and leave n_cur (the next step scatters)
};

// ---- ensembles of simulations (one batch: many independent runs advanced together) ----------
// Every simulation keeps the single-run layout -- its own control block, particle segments,
// cells and nodes -- inside arrays shared by the batch: the particles of species s of
// simulation k occupy slots [seg, seg + cap) of the batch's species arrays, its cells
// [cbase, cbase + N) of the cell arrays and its nodes [nbase, nbase + N + 1) of the node arrays.
// Cell indices stored with the particles are the simulation's own (0 .. N-1).
#define PIC_BATCH_MAX 4096  // simulations per batch

// What the batch step kernel needs of one simulation in its particle loop.
struct BSim {
  unsigned seg[2];          // first slot of each species segment in the batch arrays
  int cbase;                // first cell in the batch cell arrays
  int N;                    // cells
  unsigned long long seed;  // run seed
  unsigned collides;        // bit s: species s takes the null-collision test (its mcc_mask)
  unsigned cap[2];          // capacity of each species segment
  unsigned pad;
};

// Batch-level device words.
struct BatchDev {
  unsigned long long step;  // step the next particle step advances
  unsigned int error;       // OR of the simulations' error bits (refreshed by the plan kernel)
  unsigned int pad;
  unsigned int claim[2];    // per species: chunks claimed in the step (zeroed by the plan kernel)
};

struct BatchStep32 {
  Species32 sp[2];              // batch arrays written (the current buffer; after a sort the other)
  Species32 src[2];             // batch arrays read (the buffer the sort step left, else sp)
  unsigned int* cursor[2];      // the step after a sort: per-cell write cursors (batch cell arrays)
  unsigned int sum_ke;          // sum the kinetic energy of the particles alive after the step
  const float2* E2;             // batch cell arrays
  unsigned int* cnt[2];
  unsigned long long* S[2];
  Phys ph;                      // constants every simulation of the batch shares (push, masses)
  const StepParams32* sims;     // per simulation, pointers offset to its segment and cells
  const BSim* hot;
  const unsigned* pre[2];       // per species: chunk prefix over the simulations (nsims + 1)
  const unsigned* ncur[2];      // per species: extent of each simulation at the step's start
  BatchDev* dev;
  int nsims;
};

struct BatchPlan {
  StepParams32* sims[2];        // per-simulation parameters of both buffers (their step is set)
  unsigned* pre[2];             // out: chunk prefix (chunks of 32 * PIC_PPT particles)
  unsigned* ncur[2];            // out: extents
  BatchDev* dev;
  int nsims;
  int advance;                  // 1: the step just completed (dev->step += 1)
};

// ---- adjoint of the collisionless step ------------------------------------------------------
struct AdjState {  // one particle state: all electrons, then all ions
  int* cell;
  float* frac;
  float* vx;
  float* vy;
  float* vz;
};

struct AdjStep {
  AdjState src, dst;               // state at step start / after the step (may be the same arrays)
  int* absorb;                     // step at which each particle is absorbed (INT_MAX: never)
  const double* E;                 // node field E^n (FP64, N + 1)
  unsigned long long* R[2];        // signed int64 fixed-point node deposits (out)
  unsigned long long* jflux_fx;    // J_flux, 2^-40 fixed point (accumulated)
  unsigned long long n0, np;       // electrons [0, n0), ions [n0, np)
  long long step;
  int N;
  int mode;                        // 0 record, 1 replay, 2 recompute (no deposit, no J_flux)
  unsigned field_mode, frozen_mask, has_B;
  float qmdt2[2], t[2][3], s[2][3];
  float dtdx, E_ext;
  double flux_dtw;                 // dt * w_electron
};

struct AdjRev {
  AdjState s0, s1;                 // tape: state at the start and at the end of step n
  const int* absorb;
  const double* E;                 // E^n
  const double* chi;               // A^{-1} psi of mu^{n+1}
  const double* mu;                // mu^{n+1} (its wall entries)
  double* mu_next;                 // mu^n (accumulated)
  double *lx, *lvx, *lvy, *lvz;    // lambda (FP64)
  unsigned long long n0, np;
  long long step;
  int N;
  unsigned field_mode, frozen_mask;
  double dx, dtdx;
  double qw[2], h[2];              // q w, q dt / 2m
  double M[2][9];                  // Boris rotation per species, row-major
  double flux_dtw;                 // weight of J_flux * dt * w_electron
};

cudaError_t launch_adj_push(const AdjStep& p, int max_grid, cudaStream_t st);
cudaError_t launch_adj_deposit0(const AdjState& s, unsigned long long n0, unsigned long long np,
                                unsigned long long* R0, unsigned long long* R1, int max_grid, cudaStream_t st);
cudaError_t launch_adj_fill(int* a, unsigned long long n, int v, cudaStream_t st);
// zero_next (may be null): N + 1 values zeroed on the way (the next mu accumulator)
cudaError_t launch_adj_field_t(const double* mu, double* rhs, int N, double dx, double* gV, int with_rhs,
                               double* zero_next, cudaStream_t st);
cudaError_t launch_adj_reverse(const AdjRev& p, int max_grid, cudaStream_t st);
cudaError_t launch_adj_tgrad(const AdjRev& p, const AdjState& s0, double* partial, int blocks, cudaStream_t st);

cudaError_t launch_field(const PoissonParams& p, cudaStream_t st);
// out[s (N+1) + j] = this handle's node deposit R_sj from its per-cell counts and weight sums
cudaError_t launch_node_deposit(const PoissonParams& p, long long* out, cudaStream_t st);
// particle decomposition: drop (mark dead) the live particles whose id % nparts != part
cudaError_t launch_keep_subset(const Species32& a0, const Species32& a1, Ctl* ctl, unsigned part, unsigned nparts,
                               cudaStream_t st);
cudaError_t launch_step32(const StepParams32& p, const StepMaps& m, int grid, cudaStream_t st);
cudaError_t launch_step64(const StepParams64& p, int grid, cudaStream_t st);
cudaError_t launch_source32(const StepParams32& p, cudaStream_t st);
cudaError_t launch_source64(const StepParams64& p, cudaStream_t st);
cudaError_t launch_load32(const StepParams32& p, const unsigned long long n[2], int profile,
                          int ppc0, int ppc1, double scale, int mode, cudaStream_t st);
cudaError_t launch_load64(const StepParams64& p, const unsigned long long n[2], int profile,
                          int ppc0, int ppc1, double scale, int mode, cudaStream_t st);
cudaError_t launch_sort32(Species32 src[2], Species32 dst[2], unsigned int* cnt[2],
                          unsigned int* cursor[2], const unsigned long long cap[2], Ctl* ctl, int N,
                          int grid, cudaStream_t st);
// the scan alone, deferred: the next step kernel (scatter mode) moves the particles
cudaError_t launch_sort_scan32(Species32 src[2], Species32 dst[2], unsigned int* cnt[2], unsigned int* cursor[2],
                               const unsigned long long cap[2], Ctl* ctl, int N, cudaStream_t st);
cudaError_t launch_step32_scatter(const StepParams32& p, const StepMaps& m, int grid, cudaStream_t st);
cudaError_t launch_diag64(const StepParams64& p, int grid, cudaStream_t st);
cudaError_t launch_diag32(const StepParams32& p, int grid, cudaStream_t st);
cudaError_t launch_diag_grid(const long long* R0, const long long* R1, int sign0, int sign1, const double* E, int N,
                             double dx, Ctl* ctl, cudaStream_t st);
// species: 0, 1 (charged: undrawn countdowns are drawn at `step`) or 2 (neutrals: plain cells)
// Device checks of a checkpoint blob (k_blob.cu): the CRC-32 register of each full 64 KB block
// from a zero register; z[k] = the register update by 2048 * 2^k zero bytes (column i: image of
// bit i).  Range checks of one species' cell words and fractions.
struct BlobCrcOps {
  uint32_t z[5][32];
};
cudaError_t launch_blob_crc(const unsigned char* p, unsigned long long nblocks, const BlobCrcOps& ops, uint32_t* out,
                            cudaStream_t st);
cudaError_t launch_blob_ranges(const unsigned char* cells, const unsigned char* fracs, unsigned long long m, int N,
                               int mcc, unsigned int* bad, cudaStream_t st);
cudaError_t launch_restore32(const int* cell, const double* frac, const double* vx, const double* vy, const double* vz,
                             const unsigned long long* id, unsigned long long n, const Species32& dst,
                             unsigned long long base, const Phys& ph, int species, unsigned long long step,
                             cudaStream_t st);
// plain path: the countdown pairs a snapshot left undrawn
cudaError_t launch_fill_pairs64(unsigned* nk, const unsigned long long* id, unsigned long long n, const Phys& ph,
                                int species, unsigned long long step, cudaStream_t st);
cudaError_t launch_philox(const uint32_t* ctr, const uint32_t* key, uint32_t* out, size_t n,
                          cudaStream_t st);
// *p = v, in stream order (v is taken at the call)
cudaError_t launch_store_u64(unsigned long long* p, unsigned long long v, cudaStream_t st);
// self-test of the bounded wait: out[0] = error bits of a wait that cannot complete, out[1] = its ns
cudaError_t launch_selftest_wait(unsigned long long* out, cudaStream_t st);
// tracked neutrals
// compact: write survivors and new neutrals compacted into p.dst (else p.dst == p.src, in place)
cudaError_t launch_neutral32(const NeutralParams& p, bool compact, int grid, cudaStream_t st);
int occupancy_neutral32();
cudaError_t launch_nload32(const Species32& dst, unsigned long long n, int ppc, int N, unsigned long long seed,
                           double vt, cudaStream_t st);
cudaError_t launch_ndiag32(const Species32& a, Ctl* ctl, float mass, int grid, cudaStream_t st);

// ensembles
int bstep32_variants();
const char* bstep32_variant_name(int v);
int bstep32_occupancy(int v);
cudaError_t launch_bstep32(int v, const BatchStep32& p, const StepMaps& m, int grid, bool scatter, cudaStream_t st);
cudaError_t launch_bplan(const BatchPlan& p, cudaStream_t st);
cudaError_t launch_field_batch(const PoissonParams* tab, int nsims, int maxN, cudaStream_t st);
// the sort scans of an ensemble (tables with defer = 1: the next step moves the particles)
cudaError_t launch_sort_scan_batch(const SortParams* tab, int nsims, int maxN, cudaStream_t st);
