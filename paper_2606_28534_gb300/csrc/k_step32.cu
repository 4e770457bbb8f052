// k_step32.cu -- the fused FP32 particle step of the PIC MC cycle (paper Sec. 2: force
// interpolation, particle mover, MC collisions, deposition to the grid) for the bounded sheath
// model of Table 3 (absorbing walls, neutral background, uniform B).
//
// One persistent launch covers both species.  A CTA takes tiles of PIC_TILE consecutive
// particles of one species (the sorted order makes a tile span few cells); each thread holds
// PIC_PPT consecutive particles loaded with 128-bit accesses, and per particle:
//   gather   E_p = (1-f) E_c + f E_{c+1} from the float2 node-pair array (one 8-byte load)
//   push     Boris rotation with uniform B; cell-local position update (FP32 fraction)
//   walls    absorbed when the new cell leaves [0, N)
//   MCC      null-collision test with one Philox4x32-10 block keyed by (id ^ seed) and counter
//            (step, COLL); candidates select elastic / excitation / ionization (electrons) or
//            charge exchange (ions); ionization appends an (e, ion) pair past the array end
//   deposit  CIC in int64 fixed point: W_r = rint(f 2^32); the CTA accumulates per-cell counts
//            and sums of W_r in shared memory over the window of cells its tile touches, then
//            flushes one global atomic per touched cell.  Node deposits follow as
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

struct PushConst {
  float qmdt2, t0, t1, t2, s0, s1, s2, mass;
};

// Gather + Boris + move.  Returns the new cell (may be outside [0, N): absorbed).
__device__ __forceinline__ int push_one(const Phys& ph, const PushConst& k, const float2* __restrict__ E2,
                                        int c, float& f, float& vx, float& vy, float& vz) {
  float E = 0.f;
  if (ph.field_mode == 0u) {
    float2 e = __ldg(E2 + c);
    E = (1.f - f) * e.x + f * e.y;
  } else if (ph.field_mode == 1u) {
    E = ph.E_ext;
  }
  float a = k.qmdt2 * E;
  float mx = vx + a, my = vy, mz = vz;
  if (ph.has_B) {
    float px = mx + (my * k.t2 - mz * k.t1);
    float py = my + (mz * k.t0 - mx * k.t2);
    float pz = mz + (mx * k.t1 - my * k.t0);
    mx += py * k.s2 - pz * k.s1;
    my += pz * k.s0 - px * k.s2;
    mz += px * k.s1 - py * k.s0;
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

// Null-collision MC of one live electron; returns 1 when it ionized (child velocities out).
__device__ __forceinline__ int mcc_electron(const Phys& ph, unsigned long long id, unsigned long long step,
                                            float& vx, float& vy, float& vz, BlockCounters* bc,
                                            float* ce, float* ci, unsigned long long* kid_e,
                                            unsigned long long* kid_i) {
  const SpConst& k = ph.sp[0];
  uint4 w = draw4(id, ph.seed, step, CH_COLL, 0u);
  if (!(u01f(w.x) < k.p_null)) return 0;
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
  if (!(r < b3)) return 0;
  float dx, dy, dz;
  iso_dir_f(w.z, w.w, dx, dy, dz);
  if (r < b1) {  // elastic, energy loss (2m/M)(1 - cos chi)
    float cchi = (vx * dx + vy * dy + vz * dz) / speed;
    float sp2 = speed * sqrtf(1.f - ph.two_m_over_M * (1.f - cchi));
    vx = sp2 * dx;
    vy = sp2 * dy;
    vz = sp2 * dz;
    atomicAdd(&bc->coll[0], 1u);
    return 0;
  }
  if (r < b2) {  // excitation, loses E_ex
    float sp2 = sqrtf(2.f * (En - ph.E_ex) / k.mass);
    vx = sp2 * dx;
    vy = sp2 * dy;
    vz = sp2 * dz;
    atomicAdd(&bc->coll[1], 1u);
    return 0;
  }
  // ionization: E - E_iz split uniformly; new ion Maxwellian at T_g
  uint4 a = draw4(id, ph.seed, step, CH_SCAT, 0u);
  uint4 b = draw4(id, ph.seed, step, CH_SCAT, 1u);
  uint4 kk = draw4(id, ph.seed, step, CH_CHILD, 0u);
  float Er = En - ph.E_iz;
  float Es = u01f(a.x) * Er;
  float Ep = Er - Es;
  float spp = sqrtf(2.f * Ep / k.mass), sps = sqrtf(2.f * Es / k.mass);
  vx = spp * dx;
  vy = spp * dy;
  vz = spp * dz;
  float d2x, d2y, d2z;
  iso_dir_f(a.y, a.z, d2x, d2y, d2z);
  ce[0] = sps * d2x;
  ce[1] = sps * d2y;
  ce[2] = sps * d2z;
  float n0, n1, n2, n3;
  box_muller_f(b.x, b.y, n0, n1);
  box_muller_f(b.z, b.w, n2, n3);
  ci[0] = ph.vt_gas * n0;
  ci[1] = ph.vt_gas * n1;
  ci[2] = ph.vt_gas * n2;
  *kid_e = (unsigned long long)kk.x | ((unsigned long long)kk.y << 32);
  *kid_i = (unsigned long long)kk.z | ((unsigned long long)kk.w << 32);
  atomicAdd(&bc->coll[2], 1u);
  return 1;
}

__device__ __forceinline__ void mcc_ion(const Phys& ph, unsigned long long id, unsigned long long step,
                                        float& vx, float& vy, float& vz, BlockCounters* bc) {
  const SpConst& k = ph.sp[1];
  uint4 w = draw4(id, ph.seed, step, CH_COLL, 0u);
  if (!(u01f(w.x) < k.p_null)) return;
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
    vx = ph.vt_gas * n0;
    vy = ph.vt_gas * n1;
    vz = ph.vt_gas * n2;
    atomicAdd(&bc->coll[3], 1u);
  }
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

__global__ void __launch_bounds__(PIC_TPB, 3) k_step32(const StepParams32 P) {
  __shared__ unsigned int h_cnt[PIC_WCAP];
  __shared__ unsigned long long h_S[PIC_WCAP];
  __shared__ int red_min[PIC_TPB / 32], red_max[PIC_TPB / 32];
  __shared__ BlockCounters bc;

  const int tid = threadIdx.x;
  if (tid < (int)(sizeof(BlockCounters) / 4)) reinterpret_cast<unsigned int*>(&bc)[tid] = 0u;
  __syncthreads();

  const unsigned long long ncur0 = P.ctl->n_cur[0], ncur1 = P.ctl->n_cur[1];
  const unsigned long long tiles0 = (ncur0 + PIC_TILE - 1) / PIC_TILE;
  const unsigned long long tiles = tiles0 + (ncur1 + PIC_TILE - 1) / PIC_TILE;
  const Phys& ph = P.ph;
  const int N = ph.N;

  for (unsigned long long t = blockIdx.x; t < tiles; t += gridDim.x) {
    const int s = (t < tiles0) ? 0 : 1;
    const unsigned long long base = (s == 0 ? t : t - tiles0) * PIC_TILE;
    const unsigned long long ncur = s == 0 ? ncur0 : ncur1;
    const unsigned long long i0 = base + (unsigned long long)tid * PIC_PPT;
    const Species32 A = s ? P.sp[1] : P.sp[0];
    unsigned int* const gcnt = s ? P.cnt[1] : P.cnt[0];
    unsigned long long* const gS = s ? P.S[1] : P.S[0];
    PushConst K;
    {
      const SpConst& K0 = ph.sp[0];
      const SpConst& K1 = ph.sp[1];
      K.qmdt2 = s ? K1.qmdt2 : K0.qmdt2;
      K.t0 = s ? K1.t[0] : K0.t[0];
      K.t1 = s ? K1.t[1] : K0.t[1];
      K.t2 = s ? K1.t[2] : K0.t[2];
      K.s0 = s ? K1.s[0] : K0.s[0];
      K.s1 = s ? K1.s[1] : K0.s[1];
      K.s2 = s ? K1.s[2] : K0.s[2];
      K.mass = s ? K1.mass : K0.mass;
    }
    const bool moves = (ph.push_mask >> s) & 1u;
    const bool collides = moves && (s == 0 ? (ph.coll_mask & 7u) != 0u : (ph.coll_mask & 8u) != 0u);

    int c[PIC_PPT];
    float f[PIC_PPT], vx[PIC_PPT], vy[PIC_PPT], vz[PIC_PPT];
    unsigned long long id[PIC_PPT];
    int mult[PIC_PPT];  // 0 dead, 1 live, 2 live electron that ionized (child at the same spot)
    const bool have = i0 < ncur;
    if (have) {
      int4 c4 = *reinterpret_cast<const int4*>(A.cell + i0);
      float4 f4 = *reinterpret_cast<const float4*>(A.frac + i0);
      float4 x4 = *reinterpret_cast<const float4*>(A.vx + i0);
      float4 y4 = *reinterpret_cast<const float4*>(A.vy + i0);
      float4 z4 = *reinterpret_cast<const float4*>(A.vz + i0);
      ulonglong2 id01 = *reinterpret_cast<const ulonglong2*>(A.id + i0);
      ulonglong2 id23 = *reinterpret_cast<const ulonglong2*>(A.id + i0 + 2);
      c[0] = c4.x; c[1] = c4.y; c[2] = c4.z; c[3] = c4.w;
      f[0] = f4.x; f[1] = f4.y; f[2] = f4.z; f[3] = f4.w;
      vx[0] = x4.x; vx[1] = x4.y; vx[2] = x4.z; vx[3] = x4.w;
      vy[0] = y4.x; vy[1] = y4.y; vy[2] = y4.z; vy[3] = y4.w;
      vz[0] = z4.x; vz[1] = z4.y; vz[2] = z4.z; vz[3] = z4.w;
      id[0] = id01.x; id[1] = id01.y; id[2] = id23.x; id[3] = id23.y;
    } else {
#pragma unroll
      for (int k = 0; k < PIC_PPT; ++k) c[k] = PIC_DEAD_CELL;
    }
    int lo = 0x7FFFFFFF, hi = -1;
#pragma unroll
    for (int k = 0; k < PIC_PPT; ++k) {
      mult[k] = 0;
      if (c[k] == PIC_DEAD_CELL) continue;
      if (moves) {
        int cn = push_one(ph, K, P.E2, c[k], f[k], vx[k], vy[k], vz[k]);
        if ((unsigned)cn >= (unsigned)N) {  // absorbed at a wall
          const int side = cn < 0 ? 0 : 1;
          atomicAdd(&bc.hits[s][side], 1u);
          atomicAdd(&bc.lost[s], 1u);
          float e = 0.5f * K.mass * (vx[k] * vx[k] + vy[k] * vy[k] + vz[k] * vz[k]);
          atomicAdd(&bc.efx[s], (unsigned long long)__double2ull_rn((double)e * 16777216.0));
          c[k] = PIC_DEAD_CELL;
          continue;
        }
        c[k] = cn;
      }
      mult[k] = 1;
      if (collides) {
        if (s == 0) {
          float ce[3], ci[3];
          unsigned long long kid_e, kid_i;
          if (mcc_electron(ph, id[k], P.step, vx[k], vy[k], vz[k], &bc, ce, ci, &kid_e, &kid_i)) {
            if (append32<0>(P, ncur0, c[k], f[k], ce, kid_e)) {
              mult[k] = 2;
              atomicAdd(&bc.born[0], 1u);
            }
            if (append32<1>(P, ncur1, c[k], f[k], ci, kid_i)) {
              unsigned wr = wr_of(f[k]);
              atomicAdd(P.cnt[1] + c[k], 1u);
              atomicAdd(P.S[1] + c[k], (unsigned long long)wr);
              atomicAdd(&bc.born[1], 1u);
            }
          }
        } else {
          mcc_ion(ph, id[k], P.step, vx[k], vy[k], vz[k], &bc);
        }
      }
      lo = min(lo, c[k]);
      hi = max(hi, c[k]);
    }
    if (have && moves) {
      *reinterpret_cast<int4*>(A.cell + i0) = make_int4(c[0], c[1], c[2], c[3]);
      *reinterpret_cast<float4*>(A.frac + i0) = make_float4(f[0], f[1], f[2], f[3]);
      *reinterpret_cast<float4*>(A.vx + i0) = make_float4(vx[0], vx[1], vx[2], vx[3]);
      *reinterpret_cast<float4*>(A.vy + i0) = make_float4(vy[0], vy[1], vy[2], vy[3]);
      *reinterpret_cast<float4*>(A.vz + i0) = make_float4(vz[0], vz[1], vz[2], vz[3]);
    }

    // ---- deposit: window of cells touched by this tile ---------------------------------------
    lo = __reduce_min_sync(0xFFFFFFFFu, lo);
    hi = __reduce_max_sync(0xFFFFFFFFu, hi);
    if ((tid & 31) == 0) {
      red_min[tid >> 5] = lo;
      red_max[tid >> 5] = hi;
    }
    __syncthreads();
    lo = red_min[0];
    hi = red_max[0];
#pragma unroll
    for (int w = 1; w < PIC_TPB / 32; ++w) {
      lo = min(lo, red_min[w]);
      hi = max(hi, red_max[w]);
    }
    const int span = hi >= lo ? min(hi - lo + 1, PIC_WCAP) : 0;
    for (int j = tid; j < span; j += PIC_TPB) {
      h_cnt[j] = 0u;
      h_S[j] = 0ull;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < PIC_PPT; ++k) {
      if (!mult[k]) continue;
      // merge equal cells inside the thread (its particles are consecutive in a sorted array)
      unsigned n = (unsigned)mult[k];
      unsigned long long sw = (unsigned long long)wr_of(f[k]) * (unsigned)mult[k];
#pragma unroll
      for (int q = k + 1; q < PIC_PPT; ++q) {
        if (mult[q] && c[q] == c[k]) {
          n += (unsigned)mult[q];
          sw += (unsigned long long)wr_of(f[q]) * (unsigned)mult[q];
          mult[q] = 0;
        }
      }
      const int j = c[k] - lo;
      if (j < PIC_WCAP) {
        atomicAdd(h_cnt + j, n);
        atomicAdd(h_S + j, sw);
      } else {
        atomicAdd(gcnt + c[k], n);
        atomicAdd(gS + c[k], sw);
      }
    }
    __syncthreads();
    for (int j = tid; j < span; j += PIC_TPB) {
      unsigned n = h_cnt[j];
      if (n) {
        atomicAdd(gcnt + lo + j, n);
        atomicAdd(gS + lo + j, h_S[j]);
      }
    }
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
  } else if (tid == 15) {
    long long q = 0;
    for (int s = 0; s < 2; ++s) q += (long long)ph.sp[s].qsign * (long long)(bc.hits[s][0] + bc.hits[s][1]);
    if (q) atomicAdd(reinterpret_cast<unsigned long long*>(&g->wall_charge), (unsigned long long)q);
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
      }
    }
  }
  __syncthreads();
  if (threadIdx.x < 2 && added[threadIdx.x]) atomicAdd(&P.ctl->n_live[threadIdx.x], (unsigned long long)added[threadIdx.x]);
  if (threadIdx.x == 0) P.ctl->source_pairs += K;
}

}  // namespace

int occupancy_step32() {
  int b = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_step32, PIC_TPB, 0) != cudaSuccess || b < 1) b = 1;
  return b;
}

cudaError_t launch_step32(const StepParams32& p, int grid, cudaStream_t st) {
  k_step32<<<grid, PIC_TPB, 0, st>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_source32(const StepParams32& p, cudaStream_t st) {
  k_source32<<<1, 256, 0, st>>>(p);
  return cudaGetLastError();
}
