// step32_common.cuh -- device pieces shared by the FP32 particle-step kernels (one simulation:
// k_step32.cu; an ensemble of simulations: k_bstep32.cu): interpolation and Boris push, the
// null-collision outcomes of Sec. 2's MC collision module, the warp-aggregated int64 deposit, the
// per-warp collision queue and the TMA staging of a chunk of particles.
#pragma once
#include "pic_internal.cuh"

namespace {


struct BlockCounters {
  unsigned int hits[2][2];
  unsigned int coll[5];
  unsigned int near_thr[2];
  unsigned int viol[2];
  unsigned int lost[2];
  unsigned int born[2];
  unsigned long long efx[2];
  unsigned long long ke[2];  // kinetic energy (ke_fx32) of particles handled out of the hot loop
};

__device__ __forceinline__ void iso_dir_f(unsigned wa, unsigned wb, float& dx, float& dy, float& dz) {
  float ua = u01f(wa), ub = u01f(wb);
  float ct = 1.f - 2.f * ua;
  float st = 2.f * sqrtf(ua * (1.f - ua));
  float sp, cp;
  sincospif(2.f * ub, &sp, &cp);
  dx = st * cp;
  dy = st * sp;
  dz = ct;
}

__device__ __forceinline__ void box_muller_f(unsigned wa, unsigned wb, float& n0, float& n1) {
  float r = sqrtf(-2.f * logf(1.f - u01f(wa)));
  float s, c;
  sincospif(2.f * u01f(wb), &s, &c);
  n0 = r * c;
  n1 = r * s;
}

// Interpolation (e = node pair of the cell) + Boris + move.  Returns the new cell (may be outside
// [0, N): absorbed).
__device__ __forceinline__ int push_one(const Phys& ph, const SpConst& k, float2 e, int c, float& f, float& vx,
                                        float& vy, float& vz) {
  float E = 0.f;
  if (ph.field_mode == 0u) {
    E = (1.f - f) * e.x + f * e.y;
  } else if (ph.field_mode == 1u) {
    E = ph.E_ext;
  }
  float a = k.qmdt2 * E;
  float mx = vx + a, my = vy, mz = vz;
  if (ph.has_B) {
    float px = mx + (my * k.t[2] - mz * k.t[1]);
    float py = my + (mz * k.t[0] - mx * k.t[2]);
    float pz = mz + (mx * k.t[1] - my * k.t[0]);
    mx += py * k.s[2] - pz * k.s[1];
    my += pz * k.s[0] - px * k.s[2];
    mz += px * k.s[1] - py * k.s[0];
  }
  vx = mx + a;
  vy = my;
  vz = mz;
  float fn = f + vx * ph.dtdx;
  float fl = floorf(fn);
  f = fn - fl;
  int cn = c + (int)fl;
  if (f >= 1.f) {  // fn slightly below an integer: the fraction rounds up to 1
    f = 0.f;
    cn += 1;
  }
  return cn;
}

__device__ __forceinline__ unsigned wr_of(float f) {
  // f in [0, 1): f * 2^32 is exact in FP32 and below 2^32 - 255
  return __float2uint_rn(f * 4294967296.0f);
}

// Append one particle past the end of species s (cw: its cell word); returns false (and counts a
// drop) when full.
template <int s>
__device__ __forceinline__ bool append32(const StepParams32& P, unsigned long long ncur, int cw, float f,
                                         const float* v, unsigned long long id) {
  unsigned long long slot = ncur + atomicAdd(&P.ctl->n_born[s], 1ull);
  if (slot >= P.cap[s]) {
    atomicAdd(&P.ctl->dropped, 1ull);
    atomicOr(&P.ctl->error, ERR_OVERFLOW);
    return false;
  }
  const Species32& a = P.sp[s];
  a.cell[slot] = cw;
  a.frac[slot] = f;
  a.vx[slot] = v[0];
  a.vy[slot] = v[1];
  a.vz[slot] = v[2];
  a.id[slot] = id;
  return true;
}

// Collision of a null-collision candidate electron (its countdown expired; w: the draw (id, step,
// COLL, 0)): selects elastic, excitation, ionization or null against u1 nu_max; ionization appends
// the new (e, ion) pair at the parent's position and deposits it.  Returns the new velocity.
__device__ __forceinline__ float4 collide_electron(const StepParams32& P, unsigned long long ncur0,
                                                unsigned long long ncur1, unsigned long long id, uint4 w, int c,
                                                float f, float vx, float vy, float vz, BlockCounters* bc) {
  const Phys& ph = P.ph;
  const SpConst& k = ph.sp[0];
  const unsigned long long step = P.step;
  atomicAdd(&bc->coll[4], 1u);
  float v2 = vx * vx + vy * vy + vz * vz;
  float speed = sqrtf(v2);
  float En = 0.5f * k.mass * v2;
  float nu_el = (ph.coll_mask & 1u) ? ph.ngs_el * speed : 0.f;
  float nu_ex = 0.f, nu_iz = 0.f;
  if ((ph.coll_mask & 2u) && En > ph.E_ex) nu_ex = ph.ngs_ex * fminf((En - ph.E_ex) * ph.inv_E_ex, 1.f) * speed;
  if ((ph.coll_mask & 4u) && En > ph.E_iz) nu_iz = ph.ngs_iz * fminf((En - ph.E_iz) * ph.inv_E_iz, 1.f) * speed;
  float b1 = nu_el, b2 = b1 + nu_ex, b3 = b2 + nu_iz;
  if (b3 > k.nu_max) atomicAdd(&bc->viol[0], 1u);
  float r = u01f(w.y) * k.nu_max;
  float tol = 1e-5f * k.nu_max;
  bool near = fabsf(r - b1) < tol || fabsf(r - b2) < tol || fabsf(r - b3) < tol;
  if ((ph.coll_mask & 2u) && fabsf(En - ph.E_ex) < 1e-5f * ph.E_ex) near = true;
  if ((ph.coll_mask & 4u) && fabsf(En - ph.E_iz) < 1e-5f * ph.E_iz) near = true;
  if (near) atomicAdd(&bc->near_thr[0], 1u);
  if (!(r < b3)) return make_float4(vx, vy, vz, 1.f);
  float dx, dy, dz;
  iso_dir_f(w.z, w.w, dx, dy, dz);
  if (r < b1) {  // elastic, energy loss (2m/M)(1 - cos chi)
    float cchi = (vx * dx + vy * dy + vz * dz) / speed;
    float sp2 = speed * sqrtf(1.f - ph.two_m_over_M * (1.f - cchi));
    atomicAdd(&bc->coll[0], 1u);
    return make_float4(sp2 * dx, sp2 * dy, sp2 * dz, 1.f);
  }
  if (r < b2) {  // excitation, loses E_ex
    float sp2 = sqrtf(2.f * (En - ph.E_ex) / k.mass);
    atomicAdd(&bc->coll[1], 1u);
    return make_float4(sp2 * dx, sp2 * dy, sp2 * dz, 1.f);
  }
  // ionization: E - E_iz split uniformly; new ion Maxwellian at T_g
  uint4 a = draw4(id, ph.seed, step, CH_SCAT, 0u);
  uint4 b = draw4(id, ph.seed, step, CH_SCAT, 1u);
  uint4 kk = draw4(id, ph.seed, step, CH_CHILD, 0u);
  float Er = En - ph.E_iz;
  float Es = u01f(a.x) * Er;
  float Ep = Er - Es;
  float spp = sqrtf(2.f * Ep / k.mass), sps = sqrtf(2.f * Es / k.mass);
  float d2x, d2y, d2z;
  iso_dir_f(a.y, a.z, d2x, d2y, d2z);
  float ce[3] = {sps * d2x, sps * d2y, sps * d2z};
  float n0, n1, n2, n3;
  box_muller_f(b.x, b.y, n0, n1);
  box_muller_f(b.z, b.w, n2, n3);
  float ci[3] = {ph.vt_gas * n0, ph.vt_gas * n1, ph.vt_gas * n2};
  atomicAdd(&bc->coll[2], 1u);
  const unsigned long long wr = wr_of(f);
  const unsigned long long ide = (unsigned long long)kk.x | ((unsigned long long)kk.y << 32);
  const unsigned long long idi = (unsigned long long)kk.z | ((unsigned long long)kk.w << 32);
  if (append32<0>(P, ncur0, created_word(ph, 0, c, ide, step), f, ce, ide)) {
    atomicAdd(P.cnt[0] + c, 1u);
    atomicAdd(P.S[0] + c, wr);
    atomicAdd(&bc->born[0], 1u);
    atomicAdd(&bc->ke[0], ke_fx32(ce[0], ce[1], ce[2], ph.sp[0].mass));
  }
  if (append32<1>(P, ncur1, created_word(ph, 1, c, idi, step), f, ci, idi)) {
    atomicAdd(P.cnt[1] + c, 1u);
    atomicAdd(P.S[1] + c, wr);
    atomicAdd(&bc->born[1], 1u);
    atomicAdd(&bc->ke[1], ke_fx32(ci[0], ci[1], ci[2], ph.sp[1].mass));
  }
  return make_float4(spp * dx, spp * dy, spp * dz, 1.f);
}

// Charge exchange of a candidate ion (w: the draw (id, step, COLL, 0)): the ion leaves with a
// Maxwellian velocity at T_g.
__device__ __forceinline__ float4 collide_ion(const Phys& ph, unsigned long long id, unsigned long long step,
                                           uint4 w, float vx, float vy, float vz, BlockCounters* bc) {
  const SpConst& k = ph.sp[1];
  atomicAdd(&bc->coll[4], 1u);
  float speed = sqrtf(vx * vx + vy * vy + vz * vz);
  float b1 = ph.ngs_cx * speed;
  if (b1 > k.nu_max) atomicAdd(&bc->viol[1], 1u);
  float r = u01f(w.y) * k.nu_max;
  if (fabsf(r - b1) < 1e-5f * k.nu_max) atomicAdd(&bc->near_thr[1], 1u);
  if (r < b1) {
    uint4 a = draw4(id, ph.seed, step, CH_SCAT, 0u);
    float n0, n1, n2, n3;
    box_muller_f(w.z, w.w, n0, n1);
    box_muller_f(a.x, a.y, n2, n3);
    atomicAdd(&bc->coll[3], 1u);
    return make_float4(ph.vt_gas * n0, ph.vt_gas * n1, ph.vt_gas * n2, 1.f);
  }
  return make_float4(vx, vy, vz, 1.f);
}

// Deposit of one warp's runs of equal cells: lanes holding the same cell combine their counts
// and right-weight sums with redux.sync, and one lane issues the global reduction.  Up to two
// distinct cells per run slot are aggregated (a sorted warp spans one or two cells); remaining
// lanes (sparse regions) reduce individually.  Sums stay exact: sw < 2^35, split at bit 20 so that
// each 32-lane 32-bit sum cannot wrap.
__device__ __forceinline__ void warp_deposit(unsigned int* __restrict__ gcnt, unsigned long long* __restrict__ gS,
                                             int key, unsigned n, unsigned long long sw) {
  const int lane = threadIdx.x & 31;
  unsigned active = __ballot_sync(0xFFFFFFFFu, key >= 0);
#pragma unroll 1
  for (int it = 0; it < 2 && active; ++it) {
    const int leader = __ffs(active) - 1;
    const int kc = __shfl_sync(0xFFFFFFFFu, key, leader);
    const bool mine = key == kc;
    const unsigned n_sum = __reduce_add_sync(0xFFFFFFFFu, mine ? n : 0u);
    const unsigned lo_sum = __reduce_add_sync(0xFFFFFFFFu, mine ? (unsigned)(sw & 0xFFFFFull) : 0u);
    const unsigned hi_sum = __reduce_add_sync(0xFFFFFFFFu, mine ? (unsigned)(sw >> 20) : 0u);
    if (lane == leader) {
      atomicAdd(gcnt + kc, n_sum);
      atomicAdd(gS + kc, ((unsigned long long)hi_sum << 20) + (unsigned long long)lo_sum);
    }
    if (mine) key = -1;
    active = __ballot_sync(0xFFFFFFFFu, key >= 0);
  }
  if (key >= 0) {
    atomicAdd(gcnt + key, n);
    atomicAdd(gS + key, sw);
  }
}

// ---- deposit of a chunk through a window of cells ---------------------------------------------
// Between sorts the electrons drift: a few steps after a sort a third to three fifths of
// consecutive electrons are in different cells, so a 128-particle chunk spreads over a few
// neighbouring cells in no order, and reducing it across the warp cell by cell takes several
// rounds and leaves many single-lane global atomics (which, in the step after a sort, many warps
// aim at one dense cell at a time).  Instead each lane adds its particles to its own shared-memory
// slots for the DW cells that end at the chunk's highest cell, and each touched cell is reduced
// across the warp once, into one global reduction per array.  Particles below the window go
// straight to global memory.  Integer sums: exact in any order.
// A window of W cells (a power of two) takes W * 256 bytes per warp: column j of lane l at
// 256 j + 8 l.
template <int W>
constexpr int window_bytes() {
  return W * 32 * 8;
}

// A lane's slot holds two words for its (at most four) particles of one cell:
//   h = count << 23 + sum of (W_r >> 16),   l = sum of (W_r & 0xFFFF).
// Over a warp (at most 128 particles) the sums of h stay below 2^23 in the low field and the counts
// below 2^8, so one 32-bit warp reduction per word is exact.
__device__ __forceinline__ void red_shared_u32(unsigned a, unsigned v) {
  asm volatile("red.shared.add.u32 [%0], %1;" ::"r"(a), "r"(v) : "memory");
}

// Zeroes this lane's slots (once per kernel; the flush re-zeroes what it reads).
template <int DW>
__device__ __forceinline__ void window_zero(unsigned slots) {
#pragma unroll
  for (int j = 0; j < DW; ++j) asm volatile("st.shared.u64 [%0], %1;" ::"r"(slots + 256u * j), "l"(0ull) : "memory");
}

// Deposits the live particles of a chunk (c[k]: cell index, -1 dead; wr[k]: right weights) through
// a window of DW cells.  slots: shared address of this lane's column 0.  cell_off is added to the
// global cell index.
template <int DW>
__device__ __forceinline__ void window_deposit(unsigned slots, const int (&c)[PIC_PPT], const unsigned (&wr)[PIC_PPT],
                                               int cell_off, unsigned int* __restrict__ gcnt,
                                               unsigned long long* __restrict__ gS) {
  int lmax = -1;
#pragma unroll
  for (int k = 0; k < PIC_PPT; ++k) lmax = max(lmax, c[k]);
  const int mx = (int)__reduce_max_sync(0xFFFFFFFFu, (unsigned)(lmax + 1)) - 1;
  if (mx < 0) return;
  const int base = mx - DW + 1;
  unsigned touched = 0u;
#pragma unroll
  for (int k = 0; k < PIC_PPT; ++k) {
    if (c[k] < 0) continue;
    if (c[k] >= base) {
      const unsigned col = (unsigned)c[k] & (DW - 1);
      const unsigned a = slots + 256u * col;
      red_shared_u32(a, (1u << 23) + (wr[k] >> 16));
      red_shared_u32(a + 4u, wr[k] & 0xFFFFu);
      touched |= 1u << col;
    } else {
      atomicAdd(gcnt + cell_off + c[k], 1u);
      atomicAdd(gS + cell_off + c[k], (unsigned long long)wr[k]);
    }
  }
  unsigned cols = __reduce_or_sync(0xFFFFFFFFu, touched);
  while (cols) {
    const int col = __ffs(cols) - 1;
    cols &= cols - 1u;
    const unsigned a = slots + 256u * (unsigned)col;
    unsigned h, l;
    asm volatile("ld.shared.v2.u32 {%0, %1}, [%2];" : "=r"(h), "=r"(l) : "r"(a) : "memory");
    asm volatile("st.shared.u64 [%0], %1;" ::"r"(a), "l"(0ull) : "memory");
    const unsigned hs = __reduce_add_sync(0xFFFFFFFFu, h);
    const unsigned ls = __reduce_add_sync(0xFFFFFFFFu, l);
    if ((threadIdx.x & 31) == 0) {
      const int cell = cell_off + base + ((col - base) & (DW - 1));
      atomicAdd(gcnt + cell, hs >> 23);
      atomicAdd(gS + cell, ((unsigned long long)(hs & 0x7FFFFFu) << 16) + (unsigned long long)ls);
    }
  }
}

constexpr int QCAP = 160;   // per-warp queue of collision candidates: species << 31 | slot (the
                            // configuration check keeps capacities below 2^31)
constexpr int QFLUSH = 32;  // the warp processes its queue once it holds more than this (a
                            // chunk adds at most 32 * PIC_PPT = 128 entries)
constexpr int CHUNK = 32 * PIC_PPT;
// stage buffer of one chunk: cell | frac | vx | vy | vz (4 B each) | id (8 B)
constexpr int STAGE_BYTES = CHUNK * (5 * 4 + 8);

// The queued particles whose null-collision countdown expired in this step, one per lane: each lane
// reloads its particle (just written by this warp, so from L2), draws (id, step, COLL, 0), applies
// the collision when the expiry is a candidate, stores the new velocity and the next countdown
// (from word 0 of the same draw) in the cell word.  About one particle in a hundred expires per
// step, so this runs every few dozen chunks, out of the streaming loop's path.  Inlined: as a
// called function its register needs made the caller save registers around every call.
__device__ __forceinline__ void flush_queue(const StepParams32& P, const unsigned* q, int qn,
                                         unsigned long long ncur0, unsigned long long ncur1, BlockCounters* bc) {
  __syncwarp();
  const int lane = threadIdx.x & 31;
  for (int base = 0; base < qn; base += 32) {
    const int e = base + lane;
    if (e >= qn) break;
    const unsigned rec = q[e];
    const int s = (int)(rec >> 31);
    const unsigned long long i = rec & 0x7FFFFFFFu;
    const Species32 A = s ? P.sp[1] : P.sp[0];
    const int cw = A.cell[i];
    const int c = cw & PIC_CELL_MASK;
    const float f = A.frac[i];
    const unsigned long long id = A.id[i];
    const float vx = A.vx[i], vy = A.vy[i], vz = A.vz[i];
    const uint4 w = draw4(id, P.ph.seed, P.step, CH_COLL, 0u);
    float4 r = make_float4(vx, vy, vz, 0.f);
    if ((unsigned)cw >> (PIC_CELL_BITS + 12)) {  // the expiry is a candidate
      r = s == 0 ? collide_electron(P, ncur0, ncur1, id, w, c, f, vx, vy, vz, bc)
                 : collide_ion(P.ph, id, P.step, w, vx, vy, vz, bc);
      A.vx[i] = r.x;
      A.vy[i] = r.y;
      A.vz[i] = r.z;
    }
    A.cell[i] = c | (int)(countdown_draw(P.ph.sp[s], w.x, &bc->near_thr[s]) << PIC_CELL_BITS);
    atomicAdd(&bc->ke[s], ke_fx32(r.x, r.y, r.z, P.ph.sp[s].mass));
  }
  __syncwarp();
}

// Lane 0 starts the bulk copies of the n particles [i0, i0 + n) (n <= CHUNK, a multiple of 4, i0
// a multiple of 4) into a stage buffer; the ids only when with_id (a step that moves particles to
// new slots: the ordinary step needs no id, a particle whose countdown expires reloads its own).
__device__ __forceinline__ void stage_issue_span(const Species32& A, unsigned i0, unsigned n, unsigned char* buf,
                                                 unsigned long long* bar, bool with_id) {
  mbar_expect_tx(bar, n * (with_id ? 28u : 20u));
  tma_load_1d(buf, A.cell + i0, n * 4u, bar);
  tma_load_1d(buf + CHUNK * 4, A.frac + i0, n * 4u, bar);
  tma_load_1d(buf + CHUNK * 8, A.vx + i0, n * 4u, bar);
  tma_load_1d(buf + CHUNK * 12, A.vy + i0, n * 4u, bar);
  tma_load_1d(buf + CHUNK * 16, A.vz + i0, n * 4u, bar);
  if (with_id) tma_load_1d(buf + CHUNK * 20, A.id + i0, n * 8u, bar);
}

// Lane 0 starts the bulk copies of chunk t (ncur particles in the species) into a stage buffer.
__device__ __forceinline__ void stage_issue(const Species32& A, unsigned t, unsigned ncur, unsigned char* buf,
                                            unsigned long long* bar, bool with_id) {
  const unsigned i0 = t * CHUNK;
  stage_issue_span(A, i0, min((unsigned)CHUNK, ncur - i0), buf, bar, with_id);
}

// The same with one 2-D tensor copy of the chunk's five 4-byte arrays (the box: 128 particles x 5
// rows, the stage's layout); the ids, when asked for, by a 1-D bulk copy.  The box always arrives
// whole: past the species' capacity TMA fills zeros, and slots past ncur are never used.
__device__ __forceinline__ void stage_issue_tmap(const CUtensorMap* map, const Species32& A, unsigned t,
                                                 unsigned ncur, unsigned char* buf, unsigned long long* bar,
                                                 bool with_id) {
  const unsigned i0 = t * CHUNK;
  const unsigned n = min((unsigned)CHUNK, ncur - i0);
  mbar_expect_tx(bar, CHUNK * 20u + (with_id ? n * 8u : 0u));
  tma_load_2d(buf, map, (int)i0, 0, bar);
  if (with_id) tma_load_1d(buf + CHUNK * 20, A.id + i0, n * 8u, bar);
}

// Adds item idx (0 <= idx < 16) of a set of counters to a simulation's control block.
__device__ __forceinline__ void counters_to_ctl(Ctl* g, const Phys& ph, const BlockCounters& bc, int idx) {
  if (idx < 4) {
    unsigned v = bc.hits[idx >> 1][idx & 1];
    if (v) atomicAdd(&g->wall_hits[idx >> 1][idx & 1], (unsigned long long)v);
  } else if (idx < 9) {
    unsigned v = bc.coll[idx - 4];
    if (v) atomicAdd(&g->coll[idx - 4], (unsigned long long)v);
  } else if (idx < 11) {
    unsigned v = bc.near_thr[idx - 9];
    if (v) atomicAdd(&g->near_thr[idx - 9], (unsigned long long)v);
  } else if (idx < 13) {
    unsigned v = bc.viol[idx - 11];
    if (v) atomicAdd(&g->viol[idx - 11], (unsigned long long)v);
  } else if (idx < 15) {
    const int s = idx - 13;
    long long dl = (long long)bc.born[s] - (long long)bc.lost[s];
    if (dl) atomicAdd(&g->n_live[s], (unsigned long long)dl);
    if (bc.born[s]) atomicAdd(&g->births[s], (unsigned long long)bc.born[s]);
    if (bc.efx[s]) atomicAdd(&g->wall_energy_fx[s], bc.efx[s]);
    if (bc.ke[s]) atomicAdd(&g->ke_acc[s], bc.ke[s]);
  } else if (idx == 15) {
    long long qq = 0;
    for (int s = 0; s < 2; ++s) qq += (long long)ph.sp[s].qsign * (long long)(bc.hits[s][0] + bc.hits[s][1]);
    if (qq) atomicAdd(reinterpret_cast<unsigned long long*>(&g->wall_charge), (unsigned long long)qq);
    unsigned ion_lost = bc.hits[1][0] + bc.hits[1][1];
    if (ion_lost) atomicAdd(&g->src_K, (unsigned long long)ion_lost);
  }
}

}  // namespace
