// k_neutral.cu -- the tracked neutrals of the D+/e/D sheath (Table 3: D+ ions absorbed at the walls
// are recycled into D neutrals) and their electron-impact ionization.
//
// One launch per step, after the particle step (which logs every ion it absorbs at a wall):
//   neutrals  each neutral alive at the step start moves in a straight line (x += v_x dt / dx, the
//             cell-local update of the charged push with no force), is lost at either wall, or
//             else ionizes with probability P = 1 - exp(-K_iz n_e(x) dt), n_e(x) interpolated
//             (CIC) from the node electron density of the last deposit: the neutral becomes an ion
//             with its position, velocity and id, and an electron is born beside it (Maxwellian
//             at T_sec); both are appended to the charged species and deposited.
//   recycling each logged ion returns with probability `recycle` as a neutral on its wall (x = 0
//             or the last FP32 fraction of the last cell), v_x inward from the flux-weighted
//             half-Maxwellian at T_rec, v_y, v_z Maxwellian.
// Draws: (neutral id, step, NIZ, 0) decides the ionization, (id, step, NIZ, 1) gives the electron's
// velocity and (id, step, NIZ, 2) its id; (ion id, step, RECYCLE, 0) decides the recycling and gives
// the velocity, (ion id, step, RECYCLE, 1) the neutral's id.
//
// A warp takes chunks of 128 neutrals, lane l the entries l, l + 32, l + 64, l + 96 (every load
// instruction reads 32 consecutive values).  A neutral's velocity and id never change, so an ordinary
// step updates the buffer in place: it writes back the cell and fraction of each survivor and marks a
// lost or ionized neutral dead (36 bytes per neutral in all); new neutrals are appended past the
// extent.  On the steps that sort the charged species (COMPACT) the survivors and new neutrals are
// instead written, compacted, into the other buffer (56 bytes per neutral), which drops the dead
// slots: a warp claims one contiguous range for all its lanes' outputs with one atomic, and the
// survivors of each of the four rounds fill a contiguous run of it.  Storage order is not
// reproducible between runs; nothing depends on it (every draw is keyed by id, every deposit is an
// exact integer sum).
#include "step32_common.cuh"

namespace {

constexpr int NT_TPB = 256;
#ifndef PIC_NEUTRAL_MINB
#define PIC_NEUTRAL_MINB 3  // resident CTAs per SM the neutral step is compiled for (80 registers; the in-place kernel spills 8 bytes)
#endif

struct NCounters {
  unsigned int lost[2];
  unsigned int recycled[2];
  unsigned int ionized;
  unsigned int near;
  unsigned int born[2];
  unsigned long long started;  // neutrals alive at the step start
  unsigned long long ke[2];    // kinetic energy of the charged particles born here (2^-24 units)
};

// Ballistic move in cell-local coordinates: the position update of push_one with v unchanged.
__device__ __forceinline__ int move_one(float dtdx, int c, float& f, float vx) {
  const float fn = f + vx * dtdx;
  const float fl = floorf(fn);
  f = fn - fl;
  int cn = c + (int)fl;
  if (f >= 1.f) {
    f = 0.f;
    cn += 1;
  }
  return cn;
}

// Append a charged particle (the ion or the electron of an ionized neutral) and deposit it.
template <int s>
__device__ __forceinline__ void born_charged(const NeutralParams& Q, unsigned long long base, int c, float f,
                                             const float* v, unsigned long long id, NCounters* bc) {
  const StepParams32& P = Q.P;
  const unsigned long long slot = base + atomicAdd(&P.ctl->n_born[s], 1ull);
  if (slot >= P.cap[s]) {
    atomicAdd(&P.ctl->dropped, 1ull);
    atomicOr(&P.ctl->error, ERR_OVERFLOW);
    return;
  }
  const Species32& a = P.sp[s];
  a.cell[slot] = created_word(P.ph, s, c, id, P.step);  // with the new particle's collision countdown
  a.frac[slot] = f;
  a.vx[slot] = v[0];
  a.vy[slot] = v[1];
  a.vz[slot] = v[2];
  a.id[slot] = id;
  atomicAdd(P.cnt[s] + c, 1u);
  atomicAdd(P.S[s] + c, (unsigned long long)wr_of(f));
  atomicAdd(&bc->born[s], 1u);
  atomicAdd(&bc->ke[s], ke_fx32(v[0], v[1], v[2], P.ph.sp[s].mass));
}

// An ionizing neutral (about one in several thousand per step): the ion it becomes and the electron
// born beside it.  Inlined: as a called function its register needs made the caller save registers
// around every call.
__device__ __forceinline__ void ionize_one(const NeutralParams& Q, unsigned long long base0, unsigned long long base1,
                                        int c, float f, float vx, float vy, float vz, unsigned long long id,
                                        NCounters* bc) {
  const Phys& ph = Q.P.ph;
  const uint4 b = draw4(id, ph.seed, Q.P.step, CH_NIZ, 1u);
  const uint4 kk = draw4(id, ph.seed, Q.P.step, CH_NIZ, 2u);
  float n0, n1, n2, n3;
  box_muller_f(b.x, b.y, n0, n1);
  box_muller_f(b.z, b.w, n2, n3);
  const float ve[3] = {Q.vt_sec * n0, Q.vt_sec * n1, Q.vt_sec * n2};
  const float vi[3] = {vx, vy, vz};
  born_charged<1>(Q, base1, c, f, vi, id, bc);
  born_charged<0>(Q, base0, c, f, ve, (unsigned long long)kk.x | ((unsigned long long)kk.y << 32), bc);
  atomicAdd(&bc->ionized, 1u);
}

// Writes the lanes' kept entries (bit r of keep: entry r) compacted, one claim per warp: entry r of
// every lane lands in one contiguous run, so each store instruction covers consecutive addresses.
template <int R>
__device__ __forceinline__ void write_kept(const NeutralParams& Q, Ctl* g, unsigned long long off, unsigned keep,
                                           const int* c, const float* f, const float* vx, const float* vy,
                                           const float* vz, const unsigned long long* id) {
  const int lane = threadIdx.x & 31;
  const unsigned below = (1u << lane) - 1u;
  unsigned bal[R];
  unsigned tot = 0u;
#pragma unroll
  for (int r = 0; r < R; ++r) {
    bal[r] = __ballot_sync(0xFFFFFFFFu, (keep >> r) & 1u);
    tot += __popc(bal[r]);
  }
  if (!tot) return;
  unsigned long long base = 0ull;
  if (lane == 0) base = atomicAdd(&g->nt_out, (unsigned long long)tot);
  base = __shfl_sync(0xFFFFFFFFu, base, 0) + off;
#pragma unroll
  for (int r = 0; r < R; ++r) {
    if ((keep >> r) & 1u) {
      const unsigned long long j = base + __popc(bal[r] & below);
      if (j < Q.cap) {
        Q.dst.cell[j] = c[r];
        Q.dst.frac[j] = f[r];
        Q.dst.vx[j] = vx[r];
        Q.dst.vy[j] = vy[r];
        Q.dst.vz[j] = vz[r];
        Q.dst.id[j] = id[r];
      } else {
        atomicAdd(&g->dropped, 1ull);
        atomicOr(&g->error, ERR_OVERFLOW);
      }
    }
    base += __popc(bal[r]);
  }
}

constexpr int NT_R = 4;                 // neutrals per lane per chunk
constexpr int NT_CHUNK = 32 * NT_R;     // a warp's chunk: lane l holds entries l, l + 32, l + 64, l + 96

template <bool COMPACT>
__global__ void __launch_bounds__(NT_TPB, PIC_NEUTRAL_MINB) k_neutral32(const __grid_constant__ NeutralParams Q) {
  __shared__ NCounters bc;
  const int tid = threadIdx.x, lane = tid & 31;
  if (tid < (int)(sizeof(NCounters) / 4)) reinterpret_cast<unsigned int*>(&bc)[tid] = 0u;
  __syncthreads();

  const StepParams32& P = Q.P;
  const Phys& ph = P.ph;
  const int N = ph.N;
  Ctl* const g = P.ctl;
  const unsigned long long ncur = g->nt_cur;
  const unsigned long long nlog = Q.P.wlog ? min(g->wlog_n, P.cap[1]) : 0ull;  // the log holds cap[1] entries
  // births of the charged species go past the extent of the buffer the particle step filled
  const unsigned long long base0 = P.scatter ? g->sort_new[0] : g->n_cur[0];
  const unsigned long long base1 = P.scatter ? g->sort_new[1] : g->n_cur[1];
  const unsigned long long gw = (unsigned long long)blockIdx.x * (NT_TPB / 32) + (tid >> 5);
  const unsigned long long nwarps = (unsigned long long)gridDim.x * (NT_TPB / 32);
  unsigned long long started = 0ull;
  const unsigned long long append_at = COMPACT ? 0ull : ncur;  // new neutrals go past the extent in place

  // ---- the neutrals alive at the step start: coalesced 4- and 8-byte loads, lane-interleaved --------
  const unsigned long long nchunks = (ncur + NT_CHUNK - 1) / NT_CHUNK;
#pragma unroll 1
  for (unsigned long long ch = gw; ch < nchunks; ch += nwarps) {
    const unsigned long long i0 = ch * NT_CHUNK + lane;
    int c[NT_R];
    float f[NT_R], vx[NT_R], vy[NT_R], vz[NT_R];
    unsigned long long id[NT_R];
#pragma unroll
    for (int r = 0; r < NT_R; ++r) {
      const unsigned long long i = i0 + 32ull * r;
      c[r] = PIC_DEAD_CELL;
      if (i < ncur) {
        c[r] = checked_cell(Q.src.cell[i], N, &g->error);
        f[r] = Q.src.frac[i];
        vx[r] = Q.src.vx[i];
        vy[r] = Q.src.vy[i];
        vz[r] = Q.src.vz[i];
        id[r] = Q.src.id[i];
      }
    }
    unsigned keep = 0u, live = 0u;
#pragma unroll
    for (int r = 0; r < NT_R; ++r) {
      if (c[r] == PIC_DEAD_CELL) continue;
      live |= 1u << r;
      ++started;
      const int cn = move_one(ph.dtdx, c[r], f[r], vx[r]);
      if ((unsigned)cn >= (unsigned)N) {  // lost at a wall
        atomicAdd(&bc.lost[cn < 0 ? 0 : 1], 1u);
        continue;
      }
      c[r] = cn;
      if (Q.ionize) {
        const float2 ne2 = __ldg(Q.NE2 + cn);
        const float ne = (1.f - f[r]) * ne2.x + f[r] * ne2.y;
        const float Pz = -expm1f(-Q.Kdt * ne);
        const float u = u01f(draw4(id[r], ph.seed, P.step, CH_NIZ, 0u).x);
        if (fabsf(u - Pz) < 1e-5f * Pz) atomicAdd(&bc.near, 1u);
        if (u < Pz) {  // the neutral becomes an ion beside a new electron
          ionize_one(Q, base0, base1, cn, f[r], vx[r], vy[r], vz[r], id[r], &bc);
          continue;
        }
      }
      keep |= 1u << r;
    }
    if (COMPACT) {
      write_kept<NT_R>(Q, g, 0ull, keep, c, f, vx, vy, vz, id);
    } else {  // in place: position of each survivor, a dead mark for the others
#pragma unroll
      for (int r = 0; r < NT_R; ++r) {
        if (!((live >> r) & 1u)) continue;
        const unsigned long long i = i0 + 32ull * r;
        const bool k = (keep >> r) & 1u;
        Q.dst.cell[i] = k ? c[r] : PIC_DEAD_CELL;
        if (k) Q.dst.frac[i] = f[r];
      }
    }
  }

  // ---- the ions the particle step absorbed: each returns as a neutral with probability recycle ------
#pragma unroll 1
  for (unsigned long long e0 = gw * 32ull; e0 < nlog; e0 += nwarps * 32ull) {
    const unsigned long long e = e0 + lane;
    int c[1];
    float f[1], vx[1], vy[1], vz[1];
    unsigned long long id[1];
    unsigned keep = 0u;
    if (e < nlog) {
      const unsigned w = Q.P.wlog[e];
      const int side = (int)(w >> 31);
      const unsigned long long ion = Q.ion_id[w & 0x7FFFFFFFu];
      const uint4 d = draw4(ion, ph.seed, P.step, CH_RECYCLE, 0u);
      if ((d.x >> 8) < Q.recycle_u24) {
        const uint4 kk = draw4(ion, ph.seed, P.step, CH_RECYCLE, 1u);
        const float a = Q.vt_rec * sqrtf(-2.f * logf(1.f - u01f(d.y)));  // flux half-Maxwellian
        float n0, n1;
        box_muller_f(d.z, d.w, n0, n1);
        c[0] = side ? N - 1 : 0;
        f[0] = side ? 0.99999994f : 0.f;
        vx[0] = side ? -a : a;
        vy[0] = Q.vt_rec * n0;
        vz[0] = Q.vt_rec * n1;
        id[0] = (unsigned long long)kk.x | ((unsigned long long)kk.y << 32);
        keep = 1u;
        atomicAdd(&bc.recycled[side], 1u);
      }
    }
    write_kept<1>(Q, g, append_at, keep, c, f, vx, vy, vz, id);
  }

#pragma unroll
  for (int o = 16; o > 0; o >>= 1) started += __shfl_down_sync(0xFFFFFFFFu, started, o);
  if (lane == 0 && started) atomicAdd(&bc.started, started);
  __syncthreads();
  if (tid == 0) {
    const long long dl = (long long)bc.recycled[0] + bc.recycled[1] - bc.lost[0] - bc.lost[1] - bc.ionized;
    if (dl) atomicAdd(&g->nt_live, (unsigned long long)dl);
    if (bc.started) atomicAdd(&g->nt_particle_steps, bc.started);
    for (int k = 0; k < 2; ++k) {
      if (bc.lost[k]) atomicAdd(&g->nt_lost[k], (unsigned long long)bc.lost[k]);
      if (bc.recycled[k]) atomicAdd(&g->nt_recycled[k], (unsigned long long)bc.recycled[k]);
      if (bc.born[k]) atomicAdd(&g->n_live[k], (unsigned long long)bc.born[k]);
      if (bc.ke[k]) atomicAdd(&g->ke_acc[k], bc.ke[k]);
    }
    if (bc.ionized) atomicAdd(&g->nt_ionized, (unsigned long long)bc.ionized);
    if (bc.near) atomicAdd(&g->nt_near, (unsigned long long)bc.near);
  }
}

// Initial neutrals (uniform, neutral_ppc per cell): neutral i has id 3 << 61 | i, its position in
// cell i / ppc from the block (id, 0, INIT, 0) and its velocity, Maxwellian at T_rec, from
// (id, 0, INIT, 1); evaluated in FP64 and rounded once, as the charged load does.
__global__ void __launch_bounds__(256) k_nload32(Species32 A, unsigned long long n, int ppc, int N,
                                                 unsigned long long seed, double vt) {
  for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (unsigned long long)gridDim.x * blockDim.x) {
    const unsigned long long id = (3ull << 61) | i;
    uint4 w = draw4(id, seed, 0ull, CH_INIT, 0u);
    int c = (int)(i / (unsigned long long)ppc);
    float f = (float)u01d(w.x);  // 24-bit: exact
    if (c >= N) {
      c = N - 1;
      f = 0.99999994f;
    }
    w = draw4(id, seed, 0ull, CH_INIT, 1u);
    const double r0 = sqrt(-2.0 * log(1.0 - u01d(w.x))), r1 = sqrt(-2.0 * log(1.0 - u01d(w.z)));
    double s0, c0, s1, c1;
    sincospi(2.0 * u01d(w.y), &s0, &c0);
    sincospi(2.0 * u01d(w.w), &s1, &c1);
    A.cell[i] = c;
    A.frac[i] = f;
    A.vx[i] = (float)(vt * r0 * c0);
    A.vy[i] = (float)(vt * r0 * s0);
    A.vz[i] = (float)(vt * r1 * c1);
    A.id[i] = id;
  }
}

// Kinetic energy of the live neutrals in the 2^-24 fixed point of the charged species (ke_fx32).
__global__ void __launch_bounds__(256) k_ndiag32(Species32 A, Ctl* ctl, float mass) {
  const unsigned long long n = ctl->nt_cur;
  unsigned long long acc = 0ull;
  for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (unsigned long long)gridDim.x * blockDim.x)
    if (A.cell[i] != PIC_DEAD_CELL) acc += ke_fx32(A.vx[i], A.vy[i], A.vz[i], mass);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xFFFFFFFFu, acc, o);
  if ((threadIdx.x & 31) == 0 && acc) atomicAdd(&ctl->nt_ke_fx, acc);
}

}  // namespace

int occupancy_neutral32() {
  int b = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_neutral32<false>, NT_TPB, 0);
  return b > 0 ? b : 1;
}

cudaError_t launch_neutral32(const NeutralParams& p, bool compact, int grid, cudaStream_t st) {
  if (compact)
    k_neutral32<true><<<grid, NT_TPB, 0, st>>>(p);
  else
    k_neutral32<false><<<grid, NT_TPB, 0, st>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_nload32(const Species32& dst, unsigned long long n, int ppc, int N, unsigned long long seed,
                           double vt, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  const unsigned long long blocks = (n + 255) / 256;
  const int grid = (int)(blocks < 152ull * 16 ? blocks : 152ull * 16);
  k_nload32<<<grid, 256, 0, st>>>(dst, n, ppc, N, seed, vt);
  return cudaGetLastError();
}

cudaError_t launch_ndiag32(const Species32& a, Ctl* ctl, float mass, int grid, cudaStream_t st) {
  k_ndiag32<<<grid, 256, 0, st>>>(a, ctl, mass);
  return cudaGetLastError();
}
