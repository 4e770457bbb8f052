// k_step32.cu -- the fused FP32 particle step of the PIC MC cycle (paper Sec. 2: force
// interpolation, particle mover, MC collisions, deposition to the grid) for the bounded sheath
// model of Table 3 (absorbing walls, neutral background, uniform B).
//
// One persistent launch covers both species.  A warp takes chunks of 32 x PIC_PPT consecutive
// particles of one species (the sorted order makes a chunk span one or two cells); each lane
// holds PIC_PPT consecutive particles loaded with 128-bit accesses, and per particle:
//   gather   E_p = (1-f) E_c + f E_{c+1} from the float2 node-pair array (one 8-byte load)
//   push     Boris rotation with uniform B; cell-local position update (FP32 fraction)
//   walls    absorbed when the new cell leaves [0, N)
//   MCC      null-collision test with one Philox4x32-10 block of (particle id, step, COLL);
//            candidates are queued per warp and then select elastic / excitation / ionization
//            (electrons) or charge exchange (ions); ionization appends an (e, ion) pair past the
//            array end
//   deposit  CIC in int64 fixed point: W_r = rint(f 2^32); per cell a particle count and a sum of
//            W_r, aggregated over the lanes of a warp that share a cell (redux.sync) and added
//            to global memory with one reduction per (warp, cell).  Node deposits follow as
//            R_j = 2^32 cnt_j - S_j + S_{j-1} in the field kernel.
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

// Append one particle past the end of species s; returns false (and counts a drop) when full.
template <int s>
__device__ __forceinline__ bool append32(const StepParams32& P, unsigned long long ncur, int c, float f,
                                         const float* v, unsigned long long id) {
  unsigned long long slot = ncur + atomicAdd(&P.ctl->n_born[s], 1ull);
  if (slot >= P.cap[s]) {
    atomicAdd(&P.ctl->dropped, 1ull);
    atomicOr(&P.ctl->error, ERR_OVERFLOW);
    return false;
  }
  const Species32& a = P.sp[s];
  a.cell[slot] = c;
  a.frac[slot] = f;
  a.vx[slot] = v[0];
  a.vy[slot] = v[1];
  a.vz[slot] = v[2];
  a.id[slot] = id;
  return true;
}

// Collision of a null-collision candidate electron (P_null test already passed): selects elastic,
// excitation, ionization or null against u1 nu_max; ionization appends the new (e, ion) pair at
// the parent's position and deposits it.  Returns the new velocity.
__device__ __forceinline__ float4 collide_electron(const StepParams32& P, unsigned long long ncur0,
                                                unsigned long long ncur1, unsigned long long id, int c,
                                                float f, float vx, float vy, float vz, BlockCounters* bc) {
  const Phys& ph = P.ph;
  const SpConst& k = ph.sp[0];
  const unsigned long long step = P.step;
  uint4 w = draw4(id, ph.seed, step, CH_COLL, 0u);
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
  if (append32<0>(P, ncur0, c, f, ce, (unsigned long long)kk.x | ((unsigned long long)kk.y << 32))) {
    atomicAdd(P.cnt[0] + c, 1u);
    atomicAdd(P.S[0] + c, wr);
    atomicAdd(&bc->born[0], 1u);
    atomicAdd(&bc->ke[0], ke_fx32(ce[0], ce[1], ce[2], ph.sp[0].mass));
  }
  if (append32<1>(P, ncur1, c, f, ci, (unsigned long long)kk.z | ((unsigned long long)kk.w << 32))) {
    atomicAdd(P.cnt[1] + c, 1u);
    atomicAdd(P.S[1] + c, wr);
    atomicAdd(&bc->born[1], 1u);
    atomicAdd(&bc->ke[1], ke_fx32(ci[0], ci[1], ci[2], ph.sp[1].mass));
  }
  return make_float4(spp * dx, spp * dy, spp * dz, 1.f);
}

// Charge exchange of a candidate ion: the ion leaves with a Maxwellian velocity at T_g.
__device__ __forceinline__ float4 collide_ion(const Phys& ph, unsigned long long id, unsigned long long step,
                                           float vx, float vy, float vz, BlockCounters* bc) {
  const SpConst& k = ph.sp[1];
  uint4 w = draw4(id, ph.seed, step, CH_COLL, 0u);
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

constexpr int QCAP = 160;   // per-warp queue of collision candidates
constexpr int QFLUSH = 32;  // the warp processes its queue once it holds more than this (a
                            // chunk adds at most 32 * PIC_PPT = 128 entries)
constexpr int NSTAGE = 2;   // chunks in flight per warp (TMA double buffer)
constexpr int CHUNK = 32 * PIC_PPT;
// stage buffer of one chunk: cell | frac | vx | vy | vz (4 B each) | id (8 B)
constexpr int STAGE_BYTES = CHUNK * (5 * 4 + 8);
constexpr int WARPS = PIC_TPB / 32;
constexpr size_t STEP_SMEM = (size_t)WARPS * (NSTAGE * STAGE_BYTES + QCAP * 8 + NSTAGE * 8);

// Collisions of the queued candidates, one per lane: each lane reloads its particle (just written
// by this warp, so from L2), applies the collision and stores the new velocity.  About one
// particle in a hundred is a candidate, so this runs every few dozen chunks and keeps the rare
// code out of the streaming loop.
__device__ __noinline__ void flush_queue(const StepParams32& P, const unsigned long long* q, int qn,
                                         unsigned long long ncur0, unsigned long long ncur1, BlockCounters* bc) {
  __syncwarp();
  const int lane = threadIdx.x & 31;
  for (int base = 0; base < qn; base += 32) {
    const int e = base + lane;
    if (e >= qn) break;
    const unsigned long long rec = q[e];
    const int s = (int)(rec >> 63);
    const unsigned long long i = rec & 0x7FFFFFFFFFFFFFFFull;
    const Species32 A = s ? P.sp[1] : P.sp[0];
    const int c = A.cell[i];
    const float f = A.frac[i];
    const unsigned long long id = A.id[i];
    const float vx = A.vx[i], vy = A.vy[i], vz = A.vz[i];
    const float4 r = s == 0 ? collide_electron(P, ncur0, ncur1, id, c, f, vx, vy, vz, bc)
                            : collide_ion(P.ph, id, P.step, vx, vy, vz, bc);
    A.vx[i] = r.x;
    A.vy[i] = r.y;
    A.vz[i] = r.z;
    atomicAdd(&bc->ke[s], ke_fx32(r.x, r.y, r.z, P.ph.sp[s].mass));
  }
  __syncwarp();
}

// Lane 0 starts the bulk copies of chunk t (ncur particles in the species) into a stage buffer.
__device__ __forceinline__ void stage_issue(const Species32& A, unsigned t, unsigned ncur, unsigned char* buf,
                                            unsigned long long* bar) {
  const unsigned i0 = t * CHUNK;
  const unsigned n = min((unsigned)CHUNK, ncur - i0);  // multiple of 4
  mbar_expect_tx(bar, n * 28u);
  tma_load_1d(buf, A.cell + i0, n * 4u, bar);
  tma_load_1d(buf + CHUNK * 4, A.frac + i0, n * 4u, bar);
  tma_load_1d(buf + CHUNK * 8, A.vx + i0, n * 4u, bar);
  tma_load_1d(buf + CHUNK * 12, A.vy + i0, n * 4u, bar);
  tma_load_1d(buf + CHUNK * 16, A.vz + i0, n * 4u, bar);
  tma_load_1d(buf + CHUNK * 20, A.id + i0, n * 8u, bar);
}

// One warp handles chunks of 32 x PIC_PPT consecutive particles of one species, strided over all
// warps of the grid; the warp's next chunk is already streaming into shared memory (TMA bulk copy
// completing on an mbarrier) while it computes the current one.  No block-wide barrier inside the
// particle loop.
__global__ void __launch_bounds__(PIC_TPB, PIC_STEP_MINB) k_step32(const __grid_constant__ StepParams32 P) {
  extern __shared__ __align__(128) unsigned char dsm[];
  __shared__ BlockCounters bc;

  const int tid = threadIdx.x;
  const int lane = tid & 31, wib = tid >> 5;
  unsigned char* const stage = dsm + (size_t)wib * NSTAGE * STAGE_BYTES;
  unsigned long long* const q =
      reinterpret_cast<unsigned long long*>(dsm + (size_t)WARPS * NSTAGE * STAGE_BYTES) + (size_t)wib * QCAP;
  unsigned long long* const bar = reinterpret_cast<unsigned long long*>(
                                      dsm + (size_t)WARPS * (NSTAGE * STAGE_BYTES + QCAP * 8)) + wib * NSTAGE;
  if (tid < (int)(sizeof(BlockCounters) / 4)) reinterpret_cast<unsigned int*>(&bc)[tid] = 0u;
  if (lane < NSTAGE) mbar_init(bar + lane, 1u);
  mbar_init_fence();
  __syncthreads();

  const unsigned below = (1u << lane) - 1u;
  int qn = 0;            // warp-uniform
  unsigned parity = 0u;  // bit st: phase parity of stage st
  bool failed = false;   // a bounded wait gave up
  const unsigned long long ncur0 = P.ctl->n_cur[0], ncur1 = P.ctl->n_cur[1];
  const unsigned gw = blockIdx.x * WARPS + wib;  // particle indices and chunk counts fit 32 bits
  const unsigned nw = gridDim.x * WARPS;
  const Phys& ph = P.ph;
  const int N = ph.N;

#pragma unroll 1
  for (int s = 0; s < 2 && !failed; ++s) {
    // species arrays and constants are read from the kernel parameters where they are used
    const unsigned ncur = (unsigned)(s ? ncur1 : ncur0);
    const unsigned chunks = (ncur + CHUNK - 1) / CHUNK;
    const Species32& A = P.sp[s];
    const SpConst& K = ph.sp[s];
    const bool moves = (ph.push_mask >> s) & 1u;
    const bool collides = moves && (s == 0 ? (ph.coll_mask & 7u) != 0u : (ph.coll_mask & 8u) != 0u);
    const unsigned long long tag = (unsigned long long)s << 63;
    unsigned long long ke_lane = 0ull;  // kinetic energy of this lane's particles that stay live

    // prologue: the warp's first NSTAGE chunks
    if (lane == 0) {
#pragma unroll
      for (int st = 0; st < NSTAGE; ++st) {
        const unsigned t = gw + st * nw;
        if (t < chunks) stage_issue(A, t, ncur, stage + st * STAGE_BYTES, bar + st);
      }
    }
    int st = 0;
#pragma unroll 1
    for (unsigned t = gw; t < chunks; t += nw) {
      if (!__all_sync(0xFFFFFFFFu, mbar_wait_bounded(bar + st, (parity >> st) & 1u))) {
        failed = true;
        break;
      }
      parity ^= 1u << st;
      const unsigned char* const buf = stage + st * STAGE_BYTES;
      const unsigned i0 = t * CHUNK + lane * PIC_PPT;
      int c[PIC_PPT];
      float f[PIC_PPT], vx[PIC_PPT], vy[PIC_PPT], vz[PIC_PPT];
      unsigned long long id[PIC_PPT];
      const bool have = i0 < ncur;
      {
        const int4 c4 = reinterpret_cast<const int4*>(buf)[lane];
        const float4 f4 = reinterpret_cast<const float4*>(buf + CHUNK * 4)[lane];
        const float4 x4 = reinterpret_cast<const float4*>(buf + CHUNK * 8)[lane];
        const float4 y4 = reinterpret_cast<const float4*>(buf + CHUNK * 12)[lane];
        const float4 z4 = reinterpret_cast<const float4*>(buf + CHUNK * 16)[lane];
        const ulonglong2 id01 = reinterpret_cast<const ulonglong2*>(buf + CHUNK * 20)[2 * lane];
        const ulonglong2 id23 = reinterpret_cast<const ulonglong2*>(buf + CHUNK * 20)[2 * lane + 1];
        c[0] = c4.x; c[1] = c4.y; c[2] = c4.z; c[3] = c4.w;
        f[0] = f4.x; f[1] = f4.y; f[2] = f4.z; f[3] = f4.w;
        vx[0] = x4.x; vx[1] = x4.y; vx[2] = x4.z; vx[3] = x4.w;
        vy[0] = y4.x; vy[1] = y4.y; vy[2] = y4.z; vy[3] = y4.w;
        vz[0] = z4.x; vz[1] = z4.y; vz[2] = z4.z; vz[3] = z4.w;
        id[0] = id01.x; id[1] = id01.y; id[2] = id23.x; id[3] = id23.y;
      }
      if (!have) {
#pragma unroll
        for (int k = 0; k < PIC_PPT; ++k) {
          c[k] = PIC_DEAD_CELL;
          id[k] = 0ull;
        }
      }
      // field node pairs of the four cells, requested first so that their latency overlaps the
      // Philox work below
      float2 e2[PIC_PPT];
#pragma unroll
      for (int k = 0; k < PIC_PPT; ++k) {
        e2[k] = make_float2(0.f, 0.f);
        if (moves && ph.field_mode == 0u && c[k] != PIC_DEAD_CELL) e2[k] = __ldg(P.E2 + c[k]);
      }
      // the stage is read: refill it with the chunk NSTAGE steps ahead
      fence_proxy_async_smem();
      __syncwarp();
      if (lane == 0) {
        const unsigned tn = t + NSTAGE * nw;
        if (tn < chunks) stage_issue(A, tn, ncur, stage + st * STAGE_BYTES, bar + st);
      }
      st = st + 1 == NSTAGE ? 0 : st + 1;

      // null-collision candidates: the draw depends only on (id, step), so the four Philox
      // blocks are independent instruction streams
      unsigned cand = 0u;
      if (collides) {
#pragma unroll
        for (int k = 0; k < PIC_PPT; ++k) {
          const uint4 w = draw4(id[k], ph.seed, P.step, CH_COLL, 0u);
          if ((w.x >> 8) < K.p_null_u24) cand |= 1u << k;
        }
      }
#pragma unroll
      for (int k = 0; k < PIC_PPT; ++k) {
        if (c[k] == PIC_DEAD_CELL) continue;
        if (moves) {
          const int cn = push_one(ph, K, e2[k], c[k], f[k], vx[k], vy[k], vz[k]);
          if ((unsigned)cn >= (unsigned)N) {  // absorbed at a wall
            const int side = cn < 0 ? 0 : 1;
            atomicAdd(&bc.hits[s][side], 1u);
            atomicAdd(&bc.lost[s], 1u);
            const float e = 0.5f * K.mass * (vx[k] * vx[k] + vy[k] * vy[k] + vz[k] * vz[k]);
            atomicAdd(&bc.efx[s], (unsigned long long)__double2ull_rn((double)e * 16777216.0));
            c[k] = PIC_DEAD_CELL;
            continue;
          }
          c[k] = cn;
        }
      }
      if (have && moves) {
        *reinterpret_cast<int4*>(A.cell + i0) = make_int4(c[0], c[1], c[2], c[3]);
        *reinterpret_cast<float4*>(A.frac + i0) = make_float4(f[0], f[1], f[2], f[3]);
        *reinterpret_cast<float4*>(A.vx + i0) = make_float4(vx[0], vx[1], vx[2], vx[3]);
        *reinterpret_cast<float4*>(A.vy + i0) = make_float4(vy[0], vy[1], vy[2], vy[3]);
        *reinterpret_cast<float4*>(A.vz + i0) = make_float4(vz[0], vz[1], vz[2], vz[3]);
      }
      // kinetic energy after the push; a candidate's is added after its collision
#pragma unroll
      for (int k = 0; k < PIC_PPT; ++k)
        if (c[k] != PIC_DEAD_CELL && !((cand >> k) & 1u)) ke_lane += ke_fx32(vx[k], vy[k], vz[k], K.mass);
      // queue the surviving candidates (their collision changes v only, not the deposit)
#pragma unroll
      for (int k = 0; k < PIC_PPT; ++k) {
        const bool qk = ((cand >> k) & 1u) && c[k] != PIC_DEAD_CELL;
        const unsigned b = __ballot_sync(0xFFFFFFFFu, qk);
        if (qk) q[qn + __popc(b & below)] = tag | (unsigned long long)(i0 + k);
        qn += __popc(b);
      }

      // ---- deposit: merge equal cells inside the thread, then across the warp -----------------
      unsigned rn[PIC_PPT];
      unsigned long long rsw[PIC_PPT];
#pragma unroll
      for (int k = 0; k < PIC_PPT; ++k) {
        const bool live = c[k] != PIC_DEAD_CELL;
        rn[k] = live ? 1u : 0u;
        rsw[k] = live ? (unsigned long long)wr_of(f[k]) : 0ull;
      }
#pragma unroll
      for (int k = 0; k < PIC_PPT; ++k) {
#pragma unroll
        for (int j = k + 1; j < PIC_PPT; ++j) {
          if (rn[k] && rn[j] && c[j] == c[k]) {
            rn[k] += rn[j];
            rsw[k] += rsw[j];
            rn[j] = 0u;
          }
        }
      }
#pragma unroll
      for (int k = 0; k < PIC_PPT; ++k) warp_deposit(P.cnt[s], P.S[s], rn[k] ? c[k] : -1, rn[k], rsw[k]);

      if (qn > QFLUSH) {
        flush_queue(P, q, qn, ncur0, ncur1, &bc);
        qn = 0;
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) ke_lane += __shfl_down_sync(0xFFFFFFFFu, ke_lane, o);
    if (lane == 0 && ke_lane) atomicAdd(&bc.ke[s], ke_lane);
  }
  if (failed) {
    // a stage never completed: report, then give the copies still in flight a bounded chance to
    // land before this CTA's shared memory is released
    if (lane == 0) atomicOr(&P.ctl->error, ERR_TIMEOUT);
    for (int k = 0; k < NSTAGE; ++k) mbar_wait_bounded(bar + k, (parity >> k) & 1u);
  } else if (qn) {
    flush_queue(P, q, qn, ncur0, ncur1, &bc);
  }

// ---- flush the block counters ----------------------------------------------------------------
  __syncthreads();
  Ctl* g = P.ctl;
  if (tid < 4) {
    unsigned v = bc.hits[tid >> 1][tid & 1];
    if (v) atomicAdd(&g->wall_hits[tid >> 1][tid & 1], (unsigned long long)v);
  } else if (tid < 9) {
    unsigned v = bc.coll[tid - 4];
    if (v) atomicAdd(&g->coll[tid - 4], (unsigned long long)v);
  } else if (tid < 11) {
    unsigned v = bc.near_thr[tid - 9];
    if (v) atomicAdd(&g->near_thr[tid - 9], (unsigned long long)v);
  } else if (tid < 13) {
    unsigned v = bc.viol[tid - 11];
    if (v) atomicAdd(&g->viol[tid - 11], (unsigned long long)v);
  } else if (tid < 15) {
    const int s = tid - 13;
    long long dl = (long long)bc.born[s] - (long long)bc.lost[s];
    if (dl) atomicAdd(&g->n_live[s], (unsigned long long)dl);
    if (bc.born[s]) atomicAdd(&g->births[s], (unsigned long long)bc.born[s]);
    if (bc.efx[s]) atomicAdd(&g->wall_energy_fx[s], bc.efx[s]);
    if (bc.ke[s]) atomicAdd(&g->ke_acc[s], bc.ke[s]);
  } else if (tid == 15) {
    long long qq = 0;
    for (int s = 0; s < 2; ++s) qq += (long long)ph.sp[s].qsign * (long long)(bc.hits[s][0] + bc.hits[s][1]);
    if (qq) atomicAdd(reinterpret_cast<unsigned long long*>(&g->wall_charge), (unsigned long long)qq);
    unsigned ion_lost = bc.hits[1][0] + bc.hits[1][1];
    if (ion_lost) atomicAdd(&g->src_K, (unsigned long long)ion_lost);
  }
}

// Pair source (one pair per ion absorbed in this step), uniform in [0, x1), Maxwellian at T_s.
// Ids: 2^63 | (step & 0x7FFFFFFF) << 32 | (2k + s); positions drawn from the electron's key.
__global__ void __launch_bounds__(256) k_source32(const StepParams32 P) {
  const Phys& ph = P.ph;
  const unsigned long long K = P.ctl->src_K;
  const unsigned long long n0 = P.ctl->n_cur[0], n1 = P.ctl->n_cur[1];
  __shared__ unsigned int added[2];
  if (threadIdx.x < 2) added[threadIdx.x] = 0u;
  __syncthreads();
  for (unsigned long long k = threadIdx.x; k < K; k += blockDim.x) {
    unsigned long long ide = (1ull << 63) | ((P.step & 0x7FFFFFFFull) << 32) | (2ull * k);
    uint4 w = draw4(ide, ph.seed, P.step, CH_SOURCE, 0u);
    float x = ph.src_x1 * u01f(w.x);
    float fl = floorf(x);
    int c = (int)fl;
    float f = x - fl;
    if (f >= 1.f) { f = 0.f; c += 1; }
    if (c >= ph.N) { c = ph.N - 1; f = 0.99999994f; }
    unsigned wr = wr_of(f);
    {
      uint4 u = draw4(ide, ph.seed, P.step, CH_SOURCE, 1u);
      float a0, a1, a2, a3;
      box_muller_f(u.x, u.y, a0, a1);
      box_muller_f(u.z, u.w, a2, a3);
      float v[3] = {ph.sp[0].vt * a0, ph.sp[0].vt * a1, ph.sp[0].vt * a2};
      if (append32<0>(P, n0, c, f, v, ide)) {
        atomicAdd(P.cnt[0] + c, 1u);
        atomicAdd(P.S[0] + c, (unsigned long long)wr);
        atomicAdd(&added[0], 1u);
        atomicAdd(&P.ctl->ke_acc[0], ke_fx32(v[0], v[1], v[2], ph.sp[0].mass));
      }
    }
    {
      uint4 u = draw4(ide + 1ull, ph.seed, P.step, CH_SOURCE, 1u);
      float a0, a1, a2, a3;
      box_muller_f(u.x, u.y, a0, a1);
      box_muller_f(u.z, u.w, a2, a3);
      float v[3] = {ph.sp[1].vt * a0, ph.sp[1].vt * a1, ph.sp[1].vt * a2};
      if (append32<1>(P, n1, c, f, v, ide + 1ull)) {
        atomicAdd(P.cnt[1] + c, 1u);
        atomicAdd(P.S[1] + c, (unsigned long long)wr);
        atomicAdd(&added[1], 1u);
        atomicAdd(&P.ctl->ke_acc[1], ke_fx32(v[0], v[1], v[2], ph.sp[1].mass));
      }
    }
  }
  __syncthreads();
  if (threadIdx.x < 2 && added[threadIdx.x]) atomicAdd(&P.ctl->n_live[threadIdx.x], (unsigned long long)added[threadIdx.x]);
  if (threadIdx.x == 0) P.ctl->source_pairs += K;
}

}  // namespace

static void step32_attrs();

int occupancy_step32() {
  step32_attrs();
  int b = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_step32, PIC_TPB, STEP_SMEM) != cudaSuccess || b < 1) b = 1;
  return b;
}

static void step32_attrs() {
  static bool done = false;
  if (!done) {
    cudaFuncSetAttribute(k_step32, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)STEP_SMEM);
    done = true;
  }
}

cudaError_t launch_step32(const StepParams32& p, int grid, cudaStream_t st) {
  step32_attrs();
  k_step32<<<grid, PIC_TPB, STEP_SMEM, st>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_source32(const StepParams32& p, cudaStream_t st) {
  k_source32<<<1, 256, 0, st>>>(p);
  return cudaGetLastError();
}
