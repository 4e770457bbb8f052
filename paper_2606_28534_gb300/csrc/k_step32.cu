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
//   MCC      null collisions by geometric countdown: the particle's countdown (bits 18..30 of its
//            cell word) steps down; when it expires the particle is queued per warp, draws one
//            Philox4x32-10 block of (particle id, step, COLL), collides if the expiry is a
//            candidate -- elastic / excitation / ionization (electrons) or charge exchange
//            (ions); ionization appends an (e, ion) pair past the array end -- and takes its next
//            countdown from the same block
//   deposit  CIC in int64 fixed point: W_r = rint(f 2^32); per cell a particle count and a sum of
//            W_r.  Each lane adds its particles to its own shared-memory slots for the window of
//            cells that ends at the chunk's highest cell; each touched cell is then reduced across
//            the warp (redux.sync) into one global reduction per array (window_deposit).  Node
//            deposits follow as R_j = 2^32 cnt_j - S_j + S_{j-1} in the field kernel.
#include "step32_common.cuh"

namespace {

static_assert(PIC_PPT == 4, "each lane moves four particles: one 128-bit access per array");
#ifndef PIC_STEP_NSTAGE
#define PIC_STEP_NSTAGE 2  // chunks in flight per warp in the ordinary step (3 measured slower)
#endif
// Per variant: TMA stages per warp and the bytes of one stage (the ordinary step stages no ids).
template <bool SCATTER>
struct StepShape {
  static constexpr int TPB = PIC_TPB;
  static constexpr int WARPS = TPB / 32;
  // the ordinary step may claim chunk segments (below); after a sort, claimed segments of 12-24
  // chunks made that step 1 % faster but left an order that made the next nine steps 3 % slower,
  // and claims of one or two chunks at a time made it 20-36 % slower
  static constexpr bool DYN = !SCATTER;
  static constexpr int NSTAGE = SCATTER ? 2 : PIC_STEP_NSTAGE;
  static constexpr int SB = SCATTER ? STAGE_BYTES : CHUNK * 20;
  // cells of the deposit window: 4 in the ordinary step, so that three CTAs per SM leave the larger
  // L1 split of the SM's memory (the field gathers hit it; 0.91 -> 0.89 ms), 8 after a sort (its
  // chunks, ten steps of drift from their order, spread wider)
  static constexpr int W = SCATTER ? 8 : 4;
  static constexpr int WB = window_bytes<W>();
  static constexpr size_t SMEM = (size_t)WARPS * (NSTAGE * SB + QCAP * 4 + WB + NSTAGE * 8);
};

// One warp handles chunks of 32 x PIC_PPT consecutive particles of one species (segments of
// consecutive chunks claimed from a grid-wide counter, or a contiguous run of chunks per warp for a
// small species; strided over the warps of the grid in the step after a sort); the warp's next
// chunk is already streaming into shared memory (a TMA tensor copy
// completing on an mbarrier) while it computes the current one.  No block-wide barrier inside the
// particle loop.
// SCATTER: the step after a sort step.  The sort scan has turned the per-cell counts of the
// previous deposit into write cursors; this step reads the particles from the buffer the sort step
// left (P.src) and writes each one, pushed and collided, to its slot in the other buffer (P.sp):
// slots of one cell are claimed with one atomic per (warp, cell) group, so that a warp's writes
// stay contiguous.  A particle absorbed in this step leaves a dead slot; births are appended past
// the filled buffer's extent (sort_new).  This replaces the separate scatter pass of the sort.
#ifndef PIC_SCATTER_MINB
#define PIC_SCATTER_MINB 2  // resident CTAs per SM of the step after a sort (under 128 registers: no spills)
#endif

template <bool SCATTER>
__global__ void __launch_bounds__(StepShape<SCATTER>::TPB, SCATTER ? PIC_SCATTER_MINB : PIC_STEP_MINB)
    k_step32(const __grid_constant__ StepParams32 P, const __grid_constant__ StepMaps M) {
  extern __shared__ __align__(128) unsigned char dsm[];
  __shared__ BlockCounters bc;
  constexpr int WARPS = StepShape<SCATTER>::WARPS;
  constexpr bool DYN = StepShape<SCATTER>::DYN;
  constexpr int NSTAGE = StepShape<SCATTER>::NSTAGE;
  __shared__ unsigned stage_t[WARPS][NSTAGE];  // claimed segments: the chunk in each stage
  constexpr int SB = StepShape<SCATTER>::SB;

  const int tid = threadIdx.x;
  const int lane = tid & 31, wib = tid >> 5;
  unsigned char* const stage = dsm + (size_t)wib * NSTAGE * SB;
  unsigned* const q = reinterpret_cast<unsigned*>(dsm + (size_t)WARPS * NSTAGE * SB) + (size_t)wib * QCAP;
  const unsigned wslots =  // this lane's deposit window slots
      smem_u32(dsm + (size_t)WARPS * (NSTAGE * SB + QCAP * 4) + (size_t)wib * StepShape<SCATTER>::WB) + lane * 8u;
  unsigned long long* const bar = reinterpret_cast<unsigned long long*>(
                                      dsm + (size_t)WARPS * (NSTAGE * SB + QCAP * 4 + StepShape<SCATTER>::WB)) + wib * NSTAGE;
  if (tid < (int)(sizeof(BlockCounters) / 4)) reinterpret_cast<unsigned int*>(&bc)[tid] = 0u;
  if (lane < NSTAGE) mbar_init(bar + lane, 1u);
  window_zero<StepShape<SCATTER>::W>(wslots);
  mbar_init_fence();
  __syncthreads();

  const unsigned below = (1u << lane) - 1u;
  int qn = 0;            // warp-uniform
  unsigned parity = 0u;  // bit st: phase parity of stage st
  bool failed = false;   // a bounded wait gave up
  const unsigned long long ncur0 = P.ctl->n_cur[0], ncur1 = P.ctl->n_cur[1];
  // births go past the extent of the buffer being written
  const unsigned long long nb0 = SCATTER ? P.ctl->sort_new[0] : ncur0;
  const unsigned long long nb1 = SCATTER ? P.ctl->sort_new[1] : ncur1;
  const unsigned gw = blockIdx.x * WARPS + wib;  // particle indices and chunk counts fit 32 bits
  const unsigned nw = gridDim.x * WARPS;
  const Phys& ph = P.ph;
  const int N = ph.N;

#pragma unroll 1
  for (int s = 0; s < 2 && !failed; ++s) {
    // species arrays and constants are read from the kernel parameters where they are used
    const unsigned ncur = (unsigned)(s ? ncur1 : ncur0);
    const unsigned chunks = (ncur + CHUNK - 1) / CHUNK;
    const Species32& A = P.sp[s];                   // written
    const Species32& Asrc = SCATTER ? P.src[s] : P.sp[s];  // read
    // the species' push constants copied out once: a dynamic index into the kernel parameters costs
    // a load at every use (1.4 % of the instructions)
    SpConst Kh;
    Kh.qmdt2 = ph.sp[s].qmdt2;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      Kh.t[i] = ph.sp[s].t[i];
      Kh.s[i] = ph.sp[s].s[i];
    }
    Kh.mass = ph.sp[s].mass;
    const SpConst& K = Kh;
    const bool moves = (ph.push_mask >> s) & 1u;
    const bool collides = (ph.mcc_mask >> s) & 1u;  // takes the null-collision countdown
    const unsigned tag = (unsigned)s << 31;
    // Chunk schedule.  An ordinary step gives each warp a contiguous run of chunks: concurrent warps
    // then work in different cells, so that the deposit's reductions from different warps rarely
    // meet on one address (on the grid stride ~50 warps deposit into one dense cell at a time).  The
    // step after a sort keeps the grid stride: its cursor claims return values, and many warps in
    // one cell overlap their latencies.
    //
    // A large species (at least 48 chunks per warp) is instead claimed in segments of seg
    // consecutive chunks from a grid-wide counter, the next segment one segment ahead (its
    // atomic's round trip overlaps the current segment), so that every warp works until the species
    // runs out: with a static run per warp the warps' end times spread over a third of the launch
    // (SMs run at different speeds, and chunks in sparse regions cost more), and the last warps
    // ran with their SMs nearly empty.  seg = chunks per warp / 5 within [12, 24]: shorter
    // segments make the counter's single address a hot spot, longer ones leave a longer tail.
    const bool dyn = DYN && chunks >= 48u * nw;
    const unsigned seg = min(24u, max(12u, chunks / (5u * nw)));
    const unsigned per = (SCATTER || dyn) ? 0u : (chunks + nw - 1) / nw;
    const unsigned t_first = dyn ? 0u : SCATTER ? gw : min(chunks, gw * per);
    const unsigned t_end = (SCATTER || dyn) ? chunks : min(chunks, t_first + per);
    const unsigned t_inc = SCATTER ? nw : 1u;
    unsigned seg_cur = 0u, seg_end = 0u, seg_nxt = 0u;  // lane 0, claimed segments
    // lane 0, claimed segments: the chunk for the stage stg (the next one of the segments, recorded
    // in the stage's slot for the warp's lanes; 0xFFFFFFFF when the species is done)
    const auto next = [&](int stg) -> unsigned {
      if (seg_cur >= seg_end) {
        seg_cur = seg_nxt;
        seg_end = min(seg_nxt + seg, chunks);
        seg_nxt = atomicAdd(&P.ctl->chunk_claim[s], seg);
      }
      const unsigned tn = seg_cur < seg_end ? seg_cur++ : 0xFFFFFFFFu;
      stage_t[wib][stg] = tn;
      return tn;
    };
    unsigned long long ke_lane = 0ull;  // kinetic energy of this lane's particles that stay live

    // lane 0: the copies of chunk t into a stage buffer: one 2-D tensor copy of its five 4-byte
    // arrays, and (in the step after a sort) a bulk copy of its ids
    const auto issue = [&](unsigned t, unsigned char* buf, unsigned long long* b) {
      stage_issue_tmap(s ? &M.tmap[1] : &M.tmap[0], Asrc, t, ncur, buf, b, SCATTER);
    };
    // prologue: the warp's first NSTAGE chunks
    if (lane == 0) {
      if (dyn) seg_nxt = atomicAdd(&P.ctl->chunk_claim[s], seg);
      unsigned t = dyn ? next(0) : t_first;
#pragma unroll
      for (int st = 0; st < NSTAGE; ++st) {
        if (t < t_end) issue(t, stage + st * SB, bar + st);
        if (st + 1 < NSTAGE) t = dyn ? next(st + 1) : t + t_inc;
      }
    }
    __syncwarp();
    int st = 0;
#pragma unroll 1
    for (unsigned t = dyn ? stage_t[wib][0] : t_first; t < t_end; t = dyn ? stage_t[wib][st] : t + t_inc) {
      if (!__all_sync(0xFFFFFFFFu, mbar_wait_bounded(bar + st, (parity >> st) & 1u))) {
        failed = true;
        break;
      }
      parity ^= 1u << st;
      const unsigned char* const buf = stage + st * SB;
      const unsigned i0 = t * CHUNK + lane * PIC_PPT;
      int c[PIC_PPT];
      float f[PIC_PPT], vx[PIC_PPT], vy[PIC_PPT], vz[PIC_PPT];
      const bool have = i0 < ncur;
      {
        const int4 c4 = reinterpret_cast<const int4*>(buf)[lane];
        const float4 f4 = reinterpret_cast<const float4*>(buf + CHUNK * 4)[lane];
        const float4 x4 = reinterpret_cast<const float4*>(buf + CHUNK * 8)[lane];
        const float4 y4 = reinterpret_cast<const float4*>(buf + CHUNK * 12)[lane];
        const float4 z4 = reinterpret_cast<const float4*>(buf + CHUNK * 16)[lane];
        c[0] = c4.x; c[1] = c4.y; c[2] = c4.z; c[3] = c4.w;
        f[0] = f4.x; f[1] = f4.y; f[2] = f4.z; f[3] = f4.w;
        vx[0] = x4.x; vx[1] = x4.y; vx[2] = x4.z; vx[3] = x4.w;
        vy[0] = y4.x; vy[1] = y4.y; vy[2] = y4.z; vy[3] = y4.w;
        vz[0] = z4.x; vz[1] = z4.y; vz[2] = z4.z; vz[3] = z4.w;

      }
      if (!have) {
#pragma unroll
        for (int k = 0; k < PIC_PPT; ++k) c[k] = PIC_DEAD_CELL;
      }
#pragma unroll
      for (int k = 0; k < PIC_PPT; ++k) c[k] = checked_cell(c[k], N, &P.ctl->error);
      // field node pairs of the four cells, requested first so that their latency overlaps the
      // slot claims and the push below
      float2 e2[PIC_PPT];
#pragma unroll
      for (int k = 0; k < PIC_PPT; ++k) {
        e2[k] = make_float2(0.f, 0.f);
        if (moves && ph.field_mode == 0u && c[k] != PIC_DEAD_CELL) e2[k] = __ldg(P.E2 + (c[k] & PIC_CELL_MASK));
      }
      // the ordinary step has read its stage: refill it with the chunk NSTAGE steps ahead (the step
      // after a sort reads the ids from it at its stores, and refills it after them)
      unsigned char* const sbuf = stage + st * SB;
      if (!SCATTER) {
        fence_proxy_async_smem();
        __syncwarp();
        if (lane == 0) {
          const unsigned tn = dyn ? next(st) : t + NSTAGE * t_inc;
          if (tn < t_end) issue(tn, sbuf, bar + st);
        }
        if (dyn) __syncwarp();  // the claimed chunk is read by every lane at the loop's end
        st = st + 1 == NSTAGE ? 0 : st + 1;
      }

      unsigned live0 = 0u;  // live at the start of the step (scatter: owns a slot)
#pragma unroll
      for (int k = 0; k < PIC_PPT; ++k) live0 |= c[k] != PIC_DEAD_CELL ? (1u << k) : 0u;
      // the step after a sort claims each particle's slot in the cell it holds at the start of the
      // step (one atomic per (warp, cell) group and particle index) before the push, so that the
      // claims' round trips overlap the push; the slots are resolved at the stores
      unsigned peers[PIC_PPT], base[PIC_PPT];
      if (SCATTER) {
#pragma unroll
        for (int k = 0; k < PIC_PPT; ++k) {
          const bool live = (live0 >> k) & 1u;
          const int cell = c[k] & PIC_CELL_MASK;
          peers[k] = __match_any_sync(0xFFFFFFFFu, live ? cell : -1);
          base[k] = 0u;
          if (live && lane == __ffs(peers[k]) - 1) base[k] = atomicAdd(P.cursor[s] + cell, (unsigned)__popc(peers[k]));
        }
      }
      unsigned cand = 0u;  // the null-collision countdown expired in this step (queued)
#pragma unroll
      for (int k = 0; k < PIC_PPT; ++k) {
        if (c[k] == PIC_DEAD_CELL) continue;
        if (moves) {
          // the cell moves by dc; a survivor's word takes dc directly (its cell stays in [0, N), so
          // nothing borrows from the countdown bits)
          const int dc = push_one(ph, K, e2[k], 0, f[k], vx[k], vy[k], vz[k]);
          const int cn = (c[k] & PIC_CELL_MASK) + dc;
          if ((unsigned)cn >= (unsigned)N) {  // absorbed at a wall
            const int side = cn < 0 ? 0 : 1;
            atomicAdd(&bc.hits[s][side], 1u);
            atomicAdd(&bc.lost[s], 1u);
            if (s == 1 && P.wlog) {  // recycling: log the ion's index in the buffer read, and its wall
              const unsigned long long e = atomicAdd(&P.ctl->wlog_n, 1ull);
              if (e < P.cap[1])
                P.wlog[e] = (i0 + (unsigned)k) | ((unsigned)side << 31);
              else
                atomicOr(&P.ctl->error, ERR_DEVICE);
            }
            const float e = 0.5f * K.mass * (vx[k] * vx[k] + vy[k] * vy[k] + vz[k] * vz[k]);
            atomicAdd(&bc.efx[s], (unsigned long long)__double2ull_rn((double)e * 16777216.0));
            c[k] = PIC_DEAD_CELL;
            continue;
          }
          c[k] += dc;
          if (collides) {  // one step less to the next null-collision draw; queued when it expires
            c[k] -= 1 << PIC_CELL_BITS;
            if ((((unsigned)c[k] >> PIC_CELL_BITS) & PIC_NEXT_KMAX) == 0u) cand |= 1u << k;
          }
        }
      }
      unsigned slot[PIC_PPT];
      if (SCATTER) {
        // each particle's slot: its group's claimed base plus its rank in the group
#pragma unroll
        for (int k = 0; k < PIC_PPT; ++k)
          slot[k] = __shfl_sync(0xFFFFFFFFu, base[k], __ffs(peers[k]) - 1) + (unsigned)__popc(peers[k] & below);
        const unsigned long long* const sid = reinterpret_cast<const unsigned long long*>(sbuf + CHUNK * 20);
#pragma unroll
        for (int k = 0; k < PIC_PPT; ++k) {
          if (!((live0 >> k) & 1u)) continue;
          const unsigned j = slot[k];
          if (j >= P.cap[s]) {  // only reachable if the counts disagree with the arrays
            atomicOr(&P.ctl->error, ERR_DEVICE);
            c[k] = PIC_DEAD_CELL;
            continue;
          }
          A.cell[j] = c[k];
          if (c[k] == PIC_DEAD_CELL) continue;  // absorbed in this step: a dead slot
          A.frac[j] = f[k];
          A.vx[j] = vx[k];
          A.vy[j] = vy[k];
          A.vz[j] = vz[k];
          A.id[j] = sid[lane * PIC_PPT + k];
        }
        // the stage is read: refill it with the chunk NSTAGE steps ahead
        fence_proxy_async_smem();
        __syncwarp();
        if (lane == 0) {
          const unsigned tn = dyn ? next(st) : t + NSTAGE * t_inc;
          if (tn < t_end) issue(tn, sbuf, bar + st);
        }
        if (dyn) __syncwarp();
        st = st + 1 == NSTAGE ? 0 : st + 1;
      } else if (have && moves) {
        *reinterpret_cast<int4*>(A.cell + i0) = make_int4(c[0], c[1], c[2], c[3]);
        *reinterpret_cast<float4*>(A.frac + i0) = make_float4(f[0], f[1], f[2], f[3]);
        *reinterpret_cast<float4*>(A.vx + i0) = make_float4(vx[0], vx[1], vx[2], vx[3]);
        *reinterpret_cast<float4*>(A.vy + i0) = make_float4(vy[0], vy[1], vy[2], vy[3]);
        *reinterpret_cast<float4*>(A.vz + i0) = make_float4(vz[0], vz[1], vz[2], vz[3]);
      }
      // kinetic energy after the push (steps that sum it); a queued particle's is added after its draw
      if (P.sum_ke) {
#pragma unroll
        for (int k = 0; k < PIC_PPT; ++k)
          if (c[k] != PIC_DEAD_CELL && !((cand >> k) & 1u)) ke_lane += ke_fx32(vx[k], vy[k], vz[k], K.mass);
      }
      // queue the particles whose countdown expired (a collision changes v only, not the deposit)
      // (the ordinary step skips the four ballots when no lane of the warp has a candidate)
      // the ordinary step sets cand only for particles that survived the push and stay live; after a
      // sort a failed slot claim can still kill one
      unsigned qmask = cand;
      if (SCATTER) {
        qmask = 0u;
#pragma unroll
        for (int k = 0; k < PIC_PPT; ++k) qmask |= ((cand >> k) & 1u) && c[k] != PIC_DEAD_CELL ? 1u << k : 0u;
      }
      if (SCATTER || __any_sync(0xFFFFFFFFu, qmask != 0u)) {
#pragma unroll
        for (int k = 0; k < PIC_PPT; ++k) {
          const bool qk = (qmask >> k) & 1u;
          const unsigned b = __ballot_sync(0xFFFFFFFFu, qk);
          if (qk) q[qn + __popc(b & below)] = tag | (SCATTER ? slot[k] : i0 + k);
          qn += __popc(b);
        }
      }

      // ---- deposit through the warp's window of cells ------------------------------------------
      {
        int cc[PIC_PPT];
        unsigned wr[PIC_PPT];
#pragma unroll
        for (int k = 0; k < PIC_PPT; ++k) {
          cc[k] = c[k] != PIC_DEAD_CELL ? c[k] & PIC_CELL_MASK : -1;
          wr[k] = wr_of(f[k]);
        }
        window_deposit<StepShape<SCATTER>::W>(wslots, cc, wr, 0, P.cnt[s], P.S[s]);
      }

      if (qn > QFLUSH) {
        flush_queue(P, q, qn, nb0, nb1, &bc);
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
    flush_queue(P, q, qn, nb0, nb1, &bc);
  }

// ---- flush the block counters ----------------------------------------------------------------
  __syncthreads();
  if (tid < 16) counters_to_ctl(P.ctl, ph, bc, tid);
  if (DYN && tid == 0) {  // every claim of this CTA is done; the last CTA resets the counters
    __threadfence();  // this CTA's claims (ordered here by the barrier) before its count
    if (atomicAdd(&P.ctl->chunk_done, 1u) == gridDim.x - 1u) {
      __threadfence();  // every CTA's claims before the reset
      atomicExch(&P.ctl->chunk_claim[0], 0u);
      atomicExch(&P.ctl->chunk_claim[1], 0u);
      atomicExch(&P.ctl->chunk_done, 0u);
    }
  }
}

// Pair source (one pair per ion absorbed in this step), uniform in [0, x1), Maxwellian at T_s.
// Ids: 2^63 | (step & 0x7FFFFFFF) << 32 | (2k + s); positions drawn from the electron's key.
// Lane k of a warp makes pair k of the warp's span; the warp claims the slots of its new particles
// with one atomic per species, and sums the live counts and kinetic energies before adding them.
constexpr int SOURCE_CTAS = 32;

// The warp's new particles of species s (this lane's when mine): slots past base, deposit, counts.
template <int s>
__device__ __forceinline__ void source_append(const StepParams32& P, unsigned long long base, bool mine, int c,
                                              float f, unsigned wr, const float* v, unsigned long long id,
                                              unsigned& added, unsigned long long& ke) {
  const unsigned lane = threadIdx.x & 31u;
  const unsigned m = __ballot_sync(0xFFFFFFFFu, mine);
  unsigned long long first = 0ull;
  if (lane == 0 && m) first = atomicAdd(&P.ctl->n_born[s], (unsigned long long)__popc(m));
  first = __shfl_sync(0xFFFFFFFFu, first, 0);
  if (!mine) return;
  const unsigned long long slot = base + first + (unsigned long long)__popc(m & ((1u << lane) - 1u));
  if (slot >= P.cap[s]) {
    atomicAdd(&P.ctl->dropped, 1ull);
    atomicOr(&P.ctl->error, ERR_OVERFLOW);
    return;
  }
  const Species32& a = P.sp[s];
  a.cell[slot] = created_word(P.ph, s, c, id, P.step);
  a.frac[slot] = f;
  a.vx[slot] = v[0];
  a.vy[slot] = v[1];
  a.vz[slot] = v[2];
  a.id[slot] = id;
  atomicAdd(P.cnt[s] + c, 1u);
  atomicAdd(P.S[s] + c, (unsigned long long)wr);
  ++added;
  ke += ke_fx32(v[0], v[1], v[2], P.ph.sp[s].mass);
}

__global__ void __launch_bounds__(256) k_source32(const StepParams32 P) {
  const Phys& ph = P.ph;
  const unsigned long long K = P.ctl->src_K;
  // births go past the extent of the buffer the step filled
  const unsigned long long n0 = P.scatter ? P.ctl->sort_new[0] : P.ctl->n_cur[0];
  const unsigned long long n1 = P.scatter ? P.ctl->sort_new[1] : P.ctl->n_cur[1];
  const unsigned lane = threadIdx.x & 31u;
  unsigned added[2] = {0u, 0u};
  unsigned long long ke[2] = {0ull, 0ull};
  const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
  for (unsigned long long kw = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x - lane; kw < K; kw += stride) {
    const unsigned long long k = kw + lane;
    const bool mine = k < K;
    const unsigned long long ide = (1ull << 63) | ((P.step & 0x7FFFFFFFull) << 32) | (2ull * k);
    int c = 0;
    float f = 0.f, ve[3] = {0.f, 0.f, 0.f}, vi[3] = {0.f, 0.f, 0.f};
    if (mine) {
      const uint4 w = draw4(ide, ph.seed, P.step, CH_SOURCE, 0u);
      const float x = ph.src_x1 * u01f(w.x);
      const float fl = floorf(x);
      c = (int)fl;
      f = x - fl;
      if (f >= 1.f) { f = 0.f; c += 1; }
      if (c >= ph.N) { c = ph.N - 1; f = 0.99999994f; }
      float a0, a1, a2, a3;
      const uint4 u = draw4(ide, ph.seed, P.step, CH_SOURCE, 1u);
      box_muller_f(u.x, u.y, a0, a1);
      box_muller_f(u.z, u.w, a2, a3);
      ve[0] = ph.sp[0].vt * a0; ve[1] = ph.sp[0].vt * a1; ve[2] = ph.sp[0].vt * a2;
      const uint4 u2 = draw4(ide + 1ull, ph.seed, P.step, CH_SOURCE, 1u);
      box_muller_f(u2.x, u2.y, a0, a1);
      box_muller_f(u2.z, u2.w, a2, a3);
      vi[0] = ph.sp[1].vt * a0; vi[1] = ph.sp[1].vt * a1; vi[2] = ph.sp[1].vt * a2;
    }
    const unsigned wr = wr_of(f);
    source_append<0>(P, n0, mine, c, f, wr, ve, ide, added[0], ke[0]);
    source_append<1>(P, n1, mine, c, f, wr, vi, ide + 1ull, added[1], ke[1]);
  }
#pragma unroll
  for (int s = 0; s < 2; ++s) {
    const unsigned a = __reduce_add_sync(0xFFFFFFFFu, added[s]);
    unsigned long long e = ke[s];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) e += __shfl_down_sync(0xFFFFFFFFu, e, o);
    if (lane == 0) {
      if (a) atomicAdd(&P.ctl->n_live[s], (unsigned long long)a);
      if (e) atomicAdd(&P.ctl->ke_acc[s], e);
    }
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) P.ctl->source_pairs += K;
}

}  // namespace

static void step32_attrs();

int occupancy_step32(bool scatter) {
  step32_attrs();
  int b = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, scatter ? k_step32<true> : k_step32<false>,
                                                    scatter ? StepShape<true>::TPB : StepShape<false>::TPB,
                                                    scatter ? StepShape<true>::SMEM : StepShape<false>::SMEM) !=
                                                        cudaSuccess ||
      b < 1)
    b = 1;
  return b;
}

static void step32_attrs() {
  static bool done = false;
  if (!done) {
    cudaFuncSetAttribute(k_step32<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)StepShape<false>::SMEM);
    cudaFuncSetAttribute(k_step32<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)StepShape<true>::SMEM);
    done = true;
  }
}

cudaError_t launch_step32(const StepParams32& p, const StepMaps& m, int grid, cudaStream_t st) {
  step32_attrs();
  k_step32<false><<<grid, StepShape<false>::TPB, StepShape<false>::SMEM, st>>>(p, m);
  return cudaGetLastError();
}

cudaError_t launch_step32_scatter(const StepParams32& p, const StepMaps& m, int grid, cudaStream_t st) {
  step32_attrs();
  k_step32<true><<<grid, StepShape<true>::TPB, StepShape<true>::SMEM, st>>>(p, m);
  return cudaGetLastError();
}

cudaError_t launch_source32(const StepParams32& p, cudaStream_t st) {
  k_source32<<<SOURCE_CTAS, 256, 0, st>>>(p);
  return cudaGetLastError();
}
