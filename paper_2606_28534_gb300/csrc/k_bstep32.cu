// k_bstep32.cu -- the FP32 particle step (paper Sec. 2: interpolation, mover, MC collisions,
// deposition) of an ensemble of independent simulations in one persistent launch, and the plan
// kernel that lays out its work.
//
// Work list.  Species s of simulation k owns the chunks [pre_s[k], pre_s[k+1]) of one list over the
// whole ensemble (chunks of 32 x PIC_PPT consecutive particles of its segment; pre_s is written by
// k_bplan from the extents after the previous step).  Warp w of the grid takes the contiguous run
// [w per, (w+1) per) of the list, so that a warp meets one or two simulations per species: it keeps
// the simulation's constants (segment, cells, seed, countdown) in shared memory, its collision queue and
// its counters, and hands the counters to the simulation's control block when it moves on.
// Per particle the arithmetic is the single-run kernel's (k_step32.cu), with the simulation's cell
// offset added for the field gather and the deposit; constants every simulation shares (push,
// masses, field mode) are kernel parameters.
//
// Shapes.  The kernel is compiled for a few (CTA size, resident CTAs per SM, TMA stages per warp)
// shapes; pic_batch_set_tuning picks one at run time (the autotuner times them).  Particles per
// thread stay at PIC_PPT = 4: one 128-bit access per array.
#include "step32_common.cuh"

namespace {

static_assert(PIC_PPT == 4, "each lane moves four particles: one 128-bit access per array");

// The simulation a warp is in, as the particle loop reads it (shared memory, one per warp: read
// where used instead of held in registers through the loop).
struct WarpSim {
  unsigned seg;    // first slot of the species segment
  unsigned nk;     // extent of the species segment
  unsigned mcc;    // 1: the species takes the null-collision countdown in this simulation
  int cbase;       // first cell
  int N;           // cells
  unsigned cap;    // capacity of the species segment
  unsigned long long seed;
};

// Shared memory of a shape: per warp NST stage buffers (the ordinary step stages no ids), the
// collision queue and the stage barriers.
template <int TPB, int NST, bool SCATTER>
struct BShape {
  static constexpr int WARPS = TPB / 32;
  static constexpr int SB = SCATTER ? STAGE_BYTES : CHUNK * 20;
  static constexpr size_t SMEM = (size_t)WARPS * (NST * SB + QCAP * 4 + NST * 8);
};

// Last k < nsims with pre[k] <= t, for t < pre[nsims]: the simulation that owns chunk t.
__device__ __forceinline__ int owner(const unsigned* __restrict__ pre, int nsims, unsigned t) {
  int lo = 0, hi = nsims;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (pre[mid] <= t)
      lo = mid;
    else
      hi = mid;
  }
  return lo;
}

// Lane 0: bulk copies of local chunk lt of species s of simulation k (arrays A) into a stage buffer.
// The ids only in the step after a sort (it moves them); the ordinary step needs none.
// One 2-D tensor copy of the chunk's five 4-byte arrays (map: the batch-wide arrays of species s
// in the buffer read), at x = the chunk's first slot in the batch (a multiple of 128: segments are
// multiples of 1024 slots, so the box stays inside the simulation's segment).
__device__ __forceinline__ void issue_chunk(const BatchStep32& B, const CUtensorMap* map, const Species32& A, int s,
                                            int k, unsigned lt, unsigned char* buf, unsigned long long* bar,
                                            bool with_id) {
  const unsigned nk = B.ncur[s][k];
  const unsigned i0 = lt * CHUNK;
  const unsigned n = min((unsigned)CHUNK, nk - i0);  // multiple of 4
  const unsigned g = B.hot[k].seg[s] + i0;
  mbar_expect_tx(bar, CHUNK * 20u + (with_id ? n * 8u : 0u));
  tma_load_2d(buf, map, (int)g, 0, bar);
  if (with_id) tma_load_1d(buf + CHUNK * 20, A.id + g, n * 8u, bar);
}

// Where births of simulation k go in species s: past the extent of the buffer being written (after
// a sort, the extent the sort scan gave the filled buffer).
__device__ __forceinline__ unsigned long long birth_base(const BatchStep32& B, int k, int s, bool scatter) {
  return scatter ? B.sims[k].ctl->sort_new[s] : (unsigned long long)B.ncur[s][k];
}

// The warp leaves simulation k: its queued collisions, the kinetic energy of its particles of
// species s and its counters go to the simulation; the counters restart from zero.
__device__ __forceinline__ void leave_sim(const BatchStep32& B, int k, int s, const unsigned* q, int qn,
                                          BlockCounters& wc, unsigned long long ke, bool run_queue, bool scatter) {
  const int lane = threadIdx.x & 31;
  if (run_queue && qn)
    flush_queue(B.sims[k], q, qn, birth_base(B, k, 0, scatter), birth_base(B, k, 1, scatter), &wc);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) ke += __shfl_down_sync(0xFFFFFFFFu, ke, o);
  if (lane == 0 && ke) atomicAdd(&wc.ke[s], ke);
  __syncwarp();
  if (lane < 16) counters_to_ctl(B.sims[k].ctl, B.ph, wc, lane);
  __syncwarp();
  if (lane < (int)(sizeof(BlockCounters) / 4)) reinterpret_cast<unsigned int*>(&wc)[lane] = 0u;
  __syncwarp();
}

// SCATTER: the step after a sort step (see k_step32.cu): read B.src, write each particle to its
// sorted slot of its simulation's segment in B.sp (cursors: the sort scan's, at the simulation's
// cell offset); B.sims then addresses the written buffer, for the collision queue and births.
template <int TPB, int MINB, int NST, bool SCATTER>
__global__ void __launch_bounds__(TPB, MINB) k_bstep32(const __grid_constant__ BatchStep32 B,
                                                              const __grid_constant__ StepMaps M) {
  constexpr int WARPS = TPB / 32;
  constexpr int SB = BShape<TPB, NST, SCATTER>::SB;
  static_assert(sizeof(BlockCounters) / 4 <= 32, "one word of the counters per lane");
  extern __shared__ __align__(128) unsigned char dsm[];
  __shared__ BlockCounters wcs[WARPS];
  __shared__ WarpSim wsm[WARPS];
  __shared__ unsigned stage_t[WARPS][NST];  // claimed segments: the chunk in each stage
  // both steps may claim chunk segments: here the step after a sort already took contiguous runs
  // (the single-run kernel keeps a grid stride there), and claimed segments made it faster without
  // slowing the steps that follow (ensemble step 5.70 -> 5.51 ms averaged over a sort cycle)
  constexpr bool DYN = true;

  const int tid = threadIdx.x;
  const int lane = tid & 31, wib = tid >> 5;
  unsigned char* const stage = dsm + (size_t)wib * NST * SB;
  unsigned* const q = reinterpret_cast<unsigned*>(dsm + (size_t)WARPS * NST * SB) + (size_t)wib * QCAP;
  unsigned long long* const bar = reinterpret_cast<unsigned long long*>(
                                      dsm + (size_t)WARPS * (NST * SB + QCAP * 4)) + wib * NST;
  BlockCounters& wc = wcs[wib];
  if (lane < (int)(sizeof(BlockCounters) / 4)) reinterpret_cast<unsigned int*>(&wc)[lane] = 0u;
  if (lane < NST) mbar_init(bar + lane, 1u);
  mbar_init_fence();
  __syncthreads();

  const unsigned below = (1u << lane) - 1u;
  const Phys& ph = B.ph;
  const int nsims = B.nsims;
  const unsigned gw = blockIdx.x * WARPS + wib;
  const unsigned nw = gridDim.x * WARPS;
  int qn = 0;            // warp-uniform
  unsigned parity = 0u;  // bit st: phase parity of stage st
  bool failed = false;   // a bounded wait gave up

#pragma unroll 1
  for (int s = 0; s < 2 && !failed; ++s) {
    const unsigned* __restrict__ pre = B.pre[s];
    const unsigned total = pre[nsims];
    // Work list schedule (both steps): a contiguous run of chunks per warp, or, from 48 chunks per
    // warp on, segments of cseg consecutive chunks claimed from a counter of the batch (the next
    // one a segment ahead), so that every warp works until the species runs out (the single-run
    // step's schedule; a static run per warp ends with SMs nearly empty).
    const bool dyn = DYN && total >= 48u * nw;
    const unsigned cseg = min(24u, max(12u, total / (5u * nw)));
    unsigned seg_cur = 0u, seg_end = 0u, seg_nxt = 0u;  // lane 0, claimed segments
    // lane 0, claimed segments: the chunk for the stage stg, recorded in the stage's slot for the
    // warp's lanes (0xFFFFFFFF when the species is done)
    const auto next = [&](int stg) -> unsigned {
      if (seg_cur >= seg_end) {
        seg_cur = seg_nxt;
        seg_end = min(seg_nxt + cseg, total);
        seg_nxt = atomicAdd(&B.dev->claim[s], cseg);
      }
      const unsigned tn = seg_cur < seg_end ? seg_cur++ : 0xFFFFFFFFu;
      stage_t[wib][stg] = tn;
      return tn;
    };
    unsigned t0, t1;
    if (dyn) {
      if (lane == 0) {
        seg_nxt = atomicAdd(&B.dev->claim[s], cseg);
        next(0);
      }
      __syncwarp();
      t0 = stage_t[wib][0];
      t1 = total;
    } else {
      const unsigned per = (total + nw - 1) / nw;
      t0 = min(total, gw * per);
      t1 = min(total, t0 + per);
    }
    if (t0 >= t1) continue;
    const Species32& A = B.sp[s];                          // written
    const Species32& Asrc = SCATTER ? B.src[s] : B.sp[s];  // read
    const SpConst& K = ph.sp[s];
    const bool moves = (ph.push_mask >> s) & 1u;
    const unsigned tag = (unsigned)s << 31;
    const int kfirst = owner(pre, nsims, t0);

    // prologue: the warp's first NST chunks
    if (lane == 0) {
      int ki = kfirst;
#pragma unroll
      for (int st = 0; st < NST; ++st) {
        const unsigned t = st == 0 ? t0 : dyn ? next(st) : t0 + st;
        if (t < t1) {
          while (pre[ki + 1] <= t) ++ki;
          issue_chunk(B, s ? &M.tmap[1] : &M.tmap[0], Asrc, s, ki, t - pre[ki], stage + st * SB, bar + st, SCATTER);
        }
      }
    }
    // the simulation being processed (warp-uniform); kend == 0 until the first one is entered.
    // mcc == 0: the species takes no null-collision countdown in this simulation.
    int kc = kfirst;
    unsigned kbeg = 0u, kend = 0u;
    WarpSim& ws = wsm[wib];
    unsigned long long ke_lane = 0ull;  // kinetic energy of this lane's particles that stay live
    int st = 0;
    __syncwarp();
#pragma unroll 1
    for (unsigned t = t0; t < t1; t = dyn ? stage_t[wib][st] : t + 1u) {
      if (t >= kend) {  // first chunk of another simulation
        if (kend) {
          leave_sim(B, kc, s, q, qn, wc, ke_lane, true, SCATTER);
          qn = 0;
          ke_lane = 0ull;
        }
        while (pre[kc + 1] <= t) ++kc;
        kbeg = pre[kc];
        kend = pre[kc + 1];
        if (lane == 0) {
          const BSim& h = B.hot[kc];
          ws.seg = h.seg[s];
          ws.nk = B.ncur[s][kc];
          ws.mcc = (h.collides >> s) & 1u;
          ws.cbase = h.cbase;
          ws.N = h.N;
          ws.cap = h.cap[s];
          ws.seed = h.seed;
        }
        __syncwarp();
      }
      if (!__all_sync(0xFFFFFFFFu, mbar_wait_bounded(bar + st, (parity >> st) & 1u))) {
        failed = true;
        break;
      }
      parity ^= 1u << st;
      const unsigned char* const buf = stage + st * SB;
      const unsigned i0 = (t - kbeg) * CHUNK + lane * PIC_PPT;  // index in the simulation's segment
      int c[PIC_PPT];
      float f[PIC_PPT], vx[PIC_PPT], vy[PIC_PPT], vz[PIC_PPT];
      const bool have = i0 < ws.nk;
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
      for (int k = 0; k < PIC_PPT; ++k) c[k] = checked_cell(c[k], ws.N, &B.sims[kc].ctl->error);
      float2 e2[PIC_PPT];
#pragma unroll
      for (int k = 0; k < PIC_PPT; ++k) {
        e2[k] = make_float2(0.f, 0.f);
        if (moves && ph.field_mode == 0u && c[k] != PIC_DEAD_CELL)
          e2[k] = __ldg(B.E2 + (ws.cbase + (c[k] & PIC_CELL_MASK)));
      }
      unsigned live0 = 0u;  // live at the start of the step (the step after a sort: owns a slot)
#pragma unroll
      for (int k = 0; k < PIC_PPT; ++k) live0 |= c[k] != PIC_DEAD_CELL ? (1u << k) : 0u;
      // the ordinary step has read its stage: refill it with the chunk NST steps ahead (the step
      // after a sort reads the start-of-step cells and the ids from it again at its stores, and
      // refills it after them)
      unsigned char* const sbuf = stage + st * SB;
      const auto refill = [&](bool with_id) {
        fence_proxy_async_smem();
        __syncwarp();
        if (lane == 0) {
          const unsigned tn = dyn ? next(st) : t + NST;
          if (tn < t1) {
            int ki = kc;  // owner of chunk tn: this simulation or a later one
            while (pre[ki + 1] <= tn) ++ki;
            issue_chunk(B, s ? &M.tmap[1] : &M.tmap[0], Asrc, s, ki, tn - pre[ki], sbuf, bar + st, with_id);
          }
        }
        if (dyn) __syncwarp();  // the claimed chunk is read by every lane at the loop's end
        st = st + 1 == NST ? 0 : st + 1;
      };
      if (!SCATTER) refill(false);

      unsigned cand = 0u;  // the null-collision countdown expired in this step (queued)
      const bool collides = ws.mcc != 0u;
      const int N = ws.N;
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
            atomicAdd(&wc.hits[s][side], 1u);
            atomicAdd(&wc.lost[s], 1u);
            const float e = 0.5f * K.mass * (vx[k] * vx[k] + vy[k] * vy[k] + vz[k] * vz[k]);
            atomicAdd(&wc.efx[s], (unsigned long long)__double2ull_rn((double)e * 16777216.0));
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
        // claim each particle's slot in the cell it held at the start of the step (one atomic per
        // (warp, cell) group and particle index; the start-of-step cells are still in the stage)
        const int cb = ws.cbase;
        const int4 c4 = reinterpret_cast<const int4*>(sbuf)[lane];
        const int c0[PIC_PPT] = {c4.x, c4.y, c4.z, c4.w};
        unsigned peers[PIC_PPT], base[PIC_PPT];
#pragma unroll
        for (int k = 0; k < PIC_PPT; ++k) {
          const bool live = (live0 >> k) & 1u;
          const int cell = cb + (c0[k] & PIC_CELL_MASK);
          peers[k] = __match_any_sync(0xFFFFFFFFu, live ? cell : -1);
          base[k] = 0u;
          if (live && lane == __ffs(peers[k]) - 1)
            base[k] = atomicAdd(B.cursor[s] + cell, (unsigned)__popc(peers[k]));
        }
#pragma unroll
        for (int k = 0; k < PIC_PPT; ++k)
          slot[k] = __shfl_sync(0xFFFFFFFFu, base[k], __ffs(peers[k]) - 1) + (unsigned)__popc(peers[k] & below);
        const unsigned long long* const sid = reinterpret_cast<const unsigned long long*>(sbuf + CHUNK * 20);
        const unsigned seg = ws.seg, cap = ws.cap;
#pragma unroll
        for (int k = 0; k < PIC_PPT; ++k) {
          if (!((live0 >> k) & 1u)) continue;
          if (slot[k] >= cap) {  // only reachable if the counts disagree with the arrays
            atomicOr(&B.sims[kc].ctl->error, ERR_DEVICE);
            c[k] = PIC_DEAD_CELL;
            continue;
          }
          const unsigned j = seg + slot[k];
          A.cell[j] = c[k];
          if (c[k] == PIC_DEAD_CELL) continue;  // absorbed in this step: a dead slot
          A.frac[j] = f[k];
          A.vx[j] = vx[k];
          A.vy[j] = vy[k];
          A.vz[j] = vz[k];
          A.id[j] = sid[lane * PIC_PPT + k];
        }
        refill(true);
      } else if (have && moves) {
        const unsigned g = ws.seg + i0;
        *reinterpret_cast<int4*>(A.cell + g) = make_int4(c[0], c[1], c[2], c[3]);
        *reinterpret_cast<float4*>(A.frac + g) = make_float4(f[0], f[1], f[2], f[3]);
        *reinterpret_cast<float4*>(A.vx + g) = make_float4(vx[0], vx[1], vx[2], vx[3]);
        *reinterpret_cast<float4*>(A.vy + g) = make_float4(vy[0], vy[1], vy[2], vy[3]);
        *reinterpret_cast<float4*>(A.vz + g) = make_float4(vz[0], vz[1], vz[2], vz[3]);
      }
      if (B.sum_ke) {
#pragma unroll
        for (int k = 0; k < PIC_PPT; ++k)
          if (c[k] != PIC_DEAD_CELL && !((cand >> k) & 1u)) ke_lane += ke_fx32(vx[k], vy[k], vz[k], K.mass);
      }
      // (the ordinary step skips the four ballots when no lane of the warp has a candidate)
      unsigned qmask = 0u;
#pragma unroll
      for (int k = 0; k < PIC_PPT; ++k) qmask |= ((cand >> k) & 1u) && c[k] != PIC_DEAD_CELL ? 1u << k : 0u;
      if (SCATTER || __any_sync(0xFFFFFFFFu, qmask != 0u)) {
#pragma unroll
        for (int k = 0; k < PIC_PPT; ++k) {
          const bool qk = SCATTER ? ((cand >> k) & 1u) && c[k] != PIC_DEAD_CELL : (qmask >> k) & 1u;
          const unsigned b = __ballot_sync(0xFFFFFFFFu, qk);
          if (qk) q[qn + __popc(b & below)] = tag | (SCATTER ? slot[k] : i0 + k);
          qn += __popc(b);
        }
      }

      unsigned rn[PIC_PPT];
      unsigned long long rsw[PIC_PPT];
#pragma unroll
      for (int k = 0; k < PIC_PPT; ++k) {
        const bool live = c[k] != PIC_DEAD_CELL;
        rn[k] = live ? 1u : 0u;
        rsw[k] = live ? (unsigned long long)wr_of(f[k]) : 0ull;
      }
      const int cbase = ws.cbase;
      if (!SCATTER) {
        // runs of equal cells inside the lane, then particle 0 across the warp; particles 1..3
        // only where a lane still has one
#pragma unroll
        for (int k = PIC_PPT - 1; k > 0; --k) {
          if (rn[k] && rn[k - 1] && ((c[k] ^ c[k - 1]) & PIC_CELL_MASK) == 0) {
            rn[k - 1] += rn[k];
            rsw[k - 1] += rsw[k];
            rn[k] = 0u;
          }
        }
        warp_deposit(B.cnt[s], B.S[s], rn[0] ? cbase + (c[0] & PIC_CELL_MASK) : -1, rn[0], rsw[0]);
        if (__any_sync(0xFFFFFFFFu, (rn[1] | rn[2] | rn[3]) != 0u)) {
#pragma unroll
          for (int k = 1; k < PIC_PPT; ++k)
            warp_deposit(B.cnt[s], B.S[s], rn[k] ? cbase + (c[k] & PIC_CELL_MASK) : -1, rn[k], rsw[k]);
        }
      } else {
#pragma unroll
        for (int k = 0; k < PIC_PPT; ++k) {
#pragma unroll
          for (int j = k + 1; j < PIC_PPT; ++j) {
            if (rn[k] && rn[j] && ((c[j] ^ c[k]) & PIC_CELL_MASK) == 0) {
              rn[k] += rn[j];
              rsw[k] += rsw[j];
              rn[j] = 0u;
            }
          }
        }
#pragma unroll
        for (int k = 0; k < PIC_PPT; ++k)
          warp_deposit(B.cnt[s], B.S[s], rn[k] ? cbase + (c[k] & PIC_CELL_MASK) : -1, rn[k], rsw[k]);
      }

      if (qn > QFLUSH) {
        flush_queue(B.sims[kc], q, qn, birth_base(B, kc, 0, SCATTER), birth_base(B, kc, 1, SCATTER), &wc);
        qn = 0;
      }
    }
    if (failed) {
      // a stage never completed: report, give the copies in flight a bounded chance to land
      // before this CTA's shared memory is released, and hand over the counters (not the queue)
      if (lane == 0) {
        atomicOr(&B.dev->error, ERR_TIMEOUT);
        atomicOr(&B.sims[kc].ctl->error, ERR_TIMEOUT);
      }
      for (int k = 0; k < NST; ++k) mbar_wait_bounded(bar + k, (parity >> k) & 1u);
      if (kend) leave_sim(B, kc, s, q, 0, wc, 0ull, false, SCATTER);
    } else if (kend) {
      leave_sim(B, kc, s, q, qn, wc, ke_lane, true, SCATTER);
      qn = 0;
    }
  }
}

// ---- plan: extents, chunk and tile prefixes, error bits, step counter (one CTA of 1024) ------
constexpr int PLAN_TPB = 1024;

// Exclusive scan of one value per thread over the CTA; tot = the sum.
__device__ __forceinline__ void block_excl_scan(unsigned& a, unsigned* wa, unsigned& tot) {
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  unsigned ia = a;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned ua = __shfl_up_sync(0xFFFFFFFFu, ia, o);
    if (lane >= o) ia += ua;
  }
  if (lane == 31) wa[w] = ia;
  __syncthreads();
  if (tid < 32) {
    unsigned va = wa[tid];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned ua = __shfl_up_sync(0xFFFFFFFFu, va, o);
      if (lane >= o) va += ua;
    }
    wa[tid] = va;  // inclusive over warps
  }
  __syncthreads();
  const unsigned ea = (w ? wa[w - 1] : 0u) + ia - a;
  tot = wa[31];
  __syncthreads();  // the warp totals are reused by the next scan
  a = ea;
}

__global__ void __launch_bounds__(PLAN_TPB) k_bplan(const BatchPlan P) {
  __shared__ unsigned wa[32];
  __shared__ unsigned err_s;
  __shared__ unsigned long long step_s;
  const int tid = threadIdx.x;
  const int n = P.nsims;
  const int per = (n + PLAN_TPB - 1) / PLAN_TPB;  // at most PIC_BATCH_MAX / PLAN_TPB = 4
  const int k0 = tid * per;
  if (tid == 0) {
    err_s = 0u;
    step_s = P.dev->step + (P.advance ? 1ull : 0ull);
  }
  __syncthreads();
  unsigned err = 0u;
#pragma unroll 1
  for (int s = 0; s < 2; ++s) {
    unsigned ext[PIC_BATCH_MAX / PLAN_TPB];
    unsigned chunks = 0u;
#pragma unroll
    for (int i = 0; i < PIC_BATCH_MAX / PLAN_TPB; ++i) {
      ext[i] = 0u;
      const int k = k0 + i;
      if (i < per && k < n) {
        const Ctl* g = P.sims[0][k].ctl;
        ext[i] = (unsigned)g->n_cur[s];
        if (s == 0) err |= g->error;
        chunks += (ext[i] + 32u * PIC_PPT - 1u) / (32u * PIC_PPT);
      }
    }
    unsigned tot_c;
    block_excl_scan(chunks, wa, tot_c);
#pragma unroll
    for (int i = 0; i < PIC_BATCH_MAX / PLAN_TPB; ++i) {
      const int k = k0 + i;
      if (i < per && k < n) {
        P.pre[s][k] = chunks;
        P.ncur[s][k] = ext[i];
        chunks += (ext[i] + 32u * PIC_PPT - 1u) / (32u * PIC_PPT);
      }
    }
    if (tid == 0) P.pre[s][n] = tot_c;
  }
  if (err) atomicOr(&err_s, err);
  for (int k = tid; k < n; k += PLAN_TPB) {
    P.sims[0][k].step = step_s;
    P.sims[1][k].step = step_s;
  }
  __syncthreads();
  if (tid == 0) {
    P.dev->step = step_s;
    if (err_s) P.dev->error |= err_s;
    P.dev->claim[0] = 0u;  // the next particle step claims its chunks from zero
    P.dev->claim[1] = 0u;
  }
}

template <int TPB, int MINB, int NST, bool SCATTER>
cudaError_t launch_variant(const BatchStep32& p, const StepMaps& m, int grid, cudaStream_t st) {
  constexpr size_t smem = BShape<TPB, NST, SCATTER>::SMEM;
  static bool done = false;
  if (!done) {
    cudaFuncSetAttribute(k_bstep32<TPB, MINB, NST, SCATTER>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
    done = true;
  }
  k_bstep32<TPB, MINB, NST, SCATTER><<<grid, TPB, smem, st>>>(p, m);
  return cudaGetLastError();
}

template <int TPB, int MINB, int NST>
int occupancy_variant() {
  constexpr size_t smem0 = BShape<TPB, NST, false>::SMEM, smem1 = BShape<TPB, NST, true>::SMEM;
  int occ[2] = {0, 0};
  cudaFuncSetAttribute(k_bstep32<TPB, MINB, NST, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem0);
  cudaFuncSetAttribute(k_bstep32<TPB, MINB, NST, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem1);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ[0], k_bstep32<TPB, MINB, NST, false>, TPB, smem0);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ[1], k_bstep32<TPB, MINB, NST, true>, TPB, smem1);
  const int b = occ[0] < occ[1] ? occ[0] : occ[1];
  return b < 1 ? 1 : b;
}

struct Variant {
  const char* name;
  cudaError_t (*launch)(const BatchStep32&, const StepMaps&, int, cudaStream_t);
  cudaError_t (*launch_scatter)(const BatchStep32&, const StepMaps&, int, cudaStream_t);
  int (*occupancy)();
};

#define BSTEP32_VARIANT(T, M, S)                                                                  \
  {"tpb" #T "_minb" #M "_stages" #S, launch_variant<T, M, S, false>, launch_variant<T, M, S, true>, \
   occupancy_variant<T, M, S>}

// (threads per CTA, CTAs per SM the registers are budgeted for, TMA stages per warp)
const Variant kVariants[] = {
    BSTEP32_VARIANT(256, 3, 2),
    BSTEP32_VARIANT(128, 6, 2),
    BSTEP32_VARIANT(256, 2, 3),
    BSTEP32_VARIANT(384, 2, 2),
};
constexpr int kNumVariants = (int)(sizeof(kVariants) / sizeof(kVariants[0]));

}  // namespace

int bstep32_variants() { return kNumVariants; }

const char* bstep32_variant_name(int v) { return v >= 0 && v < kNumVariants ? kVariants[v].name : nullptr; }

int bstep32_occupancy(int v) { return v >= 0 && v < kNumVariants ? kVariants[v].occupancy() : 0; }

cudaError_t launch_bstep32(int v, const BatchStep32& p, const StepMaps& m, int grid, bool scatter, cudaStream_t st) {
  if (v < 0 || v >= kNumVariants || grid < 1) return cudaErrorInvalidValue;
  return scatter ? kVariants[v].launch_scatter(p, m, grid, st) : kVariants[v].launch(p, m, grid, st);
}

cudaError_t launch_bplan(const BatchPlan& p, cudaStream_t st) {
  if (p.nsims < 1 || p.nsims > PIC_BATCH_MAX) return cudaErrorInvalidValue;
  k_bplan<<<1, PLAN_TPB, 0, st>>>(p);
  return cudaGetLastError();
}
