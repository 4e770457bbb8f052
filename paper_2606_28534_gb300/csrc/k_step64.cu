// k_step64.cu -- the plain FP64 particle step, the baseline the FP32 path is measured against.
//
// Same method and the same random draws as the FP32 step (paper Sec. 2: interpolation, mover,
// MC collisions, deposition), written the plain way: one thread per particle over an unsorted
// array, absolute positions in cell units (FP64), the node field read from global memory, and
// the CIC deposit done with FP64 atomic adds of (1 - f) and f into per-node accumulators.  The
// null-collision countdown pair of each particle lives in its own array (nk).
#include "pic_internal.cuh"

namespace {

struct Counters64 {
  unsigned int hits[2][2];
  unsigned int coll[5];
  unsigned int near_thr[2];
  unsigned int viol[2];
  unsigned int lost[2];
  unsigned int born[2];
  unsigned long long efx[2];
};

__device__ __forceinline__ void iso_dir_d(unsigned wa, unsigned wb, double* d) {
  double ua = u01d(wa), ub = u01d(wb);
  double st = 2.0 * sqrt(ua * (1.0 - ua));
  double sp, cp;
  sincospi(2.0 * ub, &sp, &cp);
  d[0] = st * cp;
  d[1] = st * sp;
  d[2] = 1.0 - 2.0 * ua;
}

__device__ __forceinline__ void box_muller_d(unsigned wa, unsigned wb, double& n0, double& n1) {
  double r = sqrt(-2.0 * log(1.0 - u01d(wa)));
  double s, c;
  sincospi(2.0 * u01d(wb), &s, &c);
  n0 = r * c;
  n1 = r * s;
}

template <int s>
__device__ __forceinline__ bool append64(const StepParams64& P, unsigned long long ncur, double x,
                                         const double* v, unsigned long long id) {  // created in this step
  unsigned long long slot = ncur + atomicAdd(&P.ctl->n_born[s], 1ull);
  if (slot >= P.cap[s]) {
    atomicAdd(&P.ctl->dropped, 1ull);
    atomicOr(&P.ctl->error, ERR_OVERFLOW);
    return false;
  }
  const Species64& a = P.sp[s];
  a.x[slot] = x;
  a.vx[slot] = v[0];
  a.vy[slot] = v[1];
  a.vz[slot] = v[2];
  a.id[slot] = id;
  a.nk[slot] = created_pair<true>(P.ph, s, id, P.step);
  return true;
}

template <int s>
__device__ __forceinline__ void deposit64(const StepParams64& P, double x) {
  double c = floor(x);
  double f = x - c;
  int ic = (int)c;
  atomicAdd(P.acc[s] + ic, 1.0 - f);
  atomicAdd(P.acc[s] + ic + 1, f);
}

template <int s>
__device__ void particle64(const StepParams64& P, unsigned long long i, unsigned long long ncur0,
                           unsigned long long ncur1, Counters64* bc) {
  const Species64& A = P.sp[s];
  const Phys& ph = P.ph;
  const SpConst& K = ph.sp[s];
  double x = A.x[i];
  if (x < 0.0) return;  // dead slot
  double v[3] = {A.vx[i], A.vy[i], A.vz[i]};
  const bool moves = (ph.push_mask >> s) & 1u;
  if (moves) {
    double E = 0.0;
    if (ph.field_mode == 0u) {
      double c = floor(x);
      double f = x - c;
      int ic = (int)c;
      E = (1.0 - f) * P.E[ic] + f * P.E[ic + 1];
    } else if (ph.field_mode == 1u) {
      E = ph.E_ext_d;
    }
    double a = K.qmdt2_d * E;
    double m[3] = {v[0] + a, v[1], v[2]};
    if (ph.has_B) {
      double p0 = m[0] + (m[1] * K.t_d[2] - m[2] * K.t_d[1]);
      double p1 = m[1] + (m[2] * K.t_d[0] - m[0] * K.t_d[2]);
      double p2 = m[2] + (m[0] * K.t_d[1] - m[1] * K.t_d[0]);
      m[0] += p1 * K.s_d[2] - p2 * K.s_d[1];
      m[1] += p2 * K.s_d[0] - p0 * K.s_d[2];
      m[2] += p0 * K.s_d[1] - p1 * K.s_d[0];
    }
    v[0] = m[0] + a;
    v[1] = m[1];
    v[2] = m[2];
    x += v[0] * ph.dtdx_d;
    if (x < 0.0 || x >= (double)ph.N) {
      atomicAdd(&bc->hits[s][x < 0.0 ? 0 : 1], 1u);
      atomicAdd(&bc->lost[s], 1u);
      double e = 0.5 * K.mass_d * (v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
      atomicAdd(&bc->efx[s], (unsigned long long)__double2ull_rn(e * 16777216.0));
      A.x[i] = -1.0;
      return;
    }
    unsigned pair = A.nk[i];
    bool expired = false;
    if ((ph.mcc_mask >> s) & 1u) {  // the null-collision countdown
      const unsigned kk = (pair & PIC_NEXT_KMAX) - 1u;
      expired = kk == 0u;
      pair = kk | (pair & PIC_NEXT_CAND);
    }
    if (expired) {
      const uint4 w = draw4(A.id[i], ph.seed, P.step, CH_COLL, 0u);
      A.nk[i] = countdown_draw_d(K, w.x, &bc->near_thr[s]);
      if (pair & PIC_NEXT_CAND) {
        atomicAdd(&bc->coll[4], 1u);
        const double numax = (double)K.nu_max;
        const double r = u01d(w.y) * numax;
        const double v2 = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
        const double speed = sqrt(v2);
        if (s == 0) {
          const double En = 0.5 * K.mass_d * v2;
          double nu_el = (ph.coll_mask & 1u) ? ph.ngs_el_d * speed : 0.0;
          double nu_ex = 0.0, nu_iz = 0.0;
          if ((ph.coll_mask & 2u) && En > ph.E_ex_d) nu_ex = ph.ngs_ex_d * fmin((En - ph.E_ex_d) / ph.E_ex_d, 1.0) * speed;
          if ((ph.coll_mask & 4u) && En > ph.E_iz_d) nu_iz = ph.ngs_iz_d * fmin((En - ph.E_iz_d) / ph.E_iz_d, 1.0) * speed;
          double b1 = nu_el, b2 = b1 + nu_ex, b3 = b2 + nu_iz;
          if (b3 > numax) atomicAdd(&bc->viol[0], 1u);
          double tol = 1e-5 * numax;
          bool near = fabs(r - b1) < tol || fabs(r - b2) < tol || fabs(r - b3) < tol;
          if ((ph.coll_mask & 2u) && fabs(En - ph.E_ex_d) < 1e-5 * ph.E_ex_d) near = true;
          if ((ph.coll_mask & 4u) && fabs(En - ph.E_iz_d) < 1e-5 * ph.E_iz_d) near = true;
          if (near) atomicAdd(&bc->near_thr[0], 1u);
          if (r < b3) {
            double d[3];
            iso_dir_d(w.z, w.w, d);
            if (r < b1) {
              double cchi = (v[0] * d[0] + v[1] * d[1] + v[2] * d[2]) / speed;
              double sp2 = speed * sqrt(1.0 - ph.two_m_over_M_d * (1.0 - cchi));
              v[0] = sp2 * d[0];
              v[1] = sp2 * d[1];
              v[2] = sp2 * d[2];
              atomicAdd(&bc->coll[0], 1u);
            } else if (r < b2) {
              double sp2 = sqrt(2.0 * (En - ph.E_ex_d) / K.mass_d);
              v[0] = sp2 * d[0];
              v[1] = sp2 * d[1];
              v[2] = sp2 * d[2];
              atomicAdd(&bc->coll[1], 1u);
            } else {
              uint4 ua = draw4(A.id[i], ph.seed, P.step, CH_SCAT, 0u);
              uint4 ub = draw4(A.id[i], ph.seed, P.step, CH_SCAT, 1u);
              uint4 kk = draw4(A.id[i], ph.seed, P.step, CH_CHILD, 0u);
              double Er = En - ph.E_iz_d;
              double Es = u01d(ua.x) * Er;
              double Ep = Er - Es;
              double spp = sqrt(2.0 * Ep / K.mass_d), sps = sqrt(2.0 * Es / K.mass_d);
              v[0] = spp * d[0];
              v[1] = spp * d[1];
              v[2] = spp * d[2];
              double d2[3];
              iso_dir_d(ua.y, ua.z, d2);
              double ce[3] = {sps * d2[0], sps * d2[1], sps * d2[2]};
              double n0, n1, n2, n3;
              box_muller_d(ub.x, ub.y, n0, n1);
              box_muller_d(ub.z, ub.w, n2, n3);
              double ci[3] = {ph.vt_gas_d * n0, ph.vt_gas_d * n1, ph.vt_gas_d * n2};
              unsigned long long kid_e = (unsigned long long)kk.x | ((unsigned long long)kk.y << 32);
              unsigned long long kid_i = (unsigned long long)kk.z | ((unsigned long long)kk.w << 32);
              if (append64<0>(P, ncur0, x, ce, kid_e)) {
                deposit64<0>(P, x);
                atomicAdd(&bc->born[0], 1u);
              }
              if (append64<1>(P, ncur1, x, ci, kid_i)) {
                deposit64<1>(P, x);
                atomicAdd(&bc->born[1], 1u);
              }
              atomicAdd(&bc->coll[2], 1u);
            }
          }
        } else {
          double b1 = ph.ngs_cx_d * speed;
          if (b1 > numax) atomicAdd(&bc->viol[1], 1u);
          if (fabs(r - b1) < 1e-5 * numax) atomicAdd(&bc->near_thr[1], 1u);
          if (r < b1) {
            uint4 ua = draw4(A.id[i], ph.seed, P.step, CH_SCAT, 0u);
            double n0, n1, n2, n3;
            box_muller_d(w.z, w.w, n0, n1);
            box_muller_d(ua.x, ua.y, n2, n3);
            v[0] = ph.vt_gas_d * n0;
            v[1] = ph.vt_gas_d * n1;
            v[2] = ph.vt_gas_d * n2;
            atomicAdd(&bc->coll[3], 1u);
          }
        }
      }
    } else if ((ph.mcc_mask >> s) & 1u) {
      A.nk[i] = pair;
    }
    A.x[i] = x;
    A.vx[i] = v[0];
    A.vy[i] = v[1];
    A.vz[i] = v[2];
  }
  deposit64<s>(P, x);
}

__global__ void __launch_bounds__(256) k_step64(const StepParams64 P) {
  __shared__ Counters64 bc;
  const int tid = threadIdx.x;
  if (tid < (int)(sizeof(Counters64) / 4)) reinterpret_cast<unsigned int*>(&bc)[tid] = 0u;
  __syncthreads();
  const unsigned long long n0 = P.ctl->n_cur[0], n1 = P.ctl->n_cur[1];
  const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
  for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + tid; i < n0 + n1; i += stride) {
    if (i < n0)
      particle64<0>(P, i, n0, n1, &bc);
    else
      particle64<1>(P, i - n0, n0, n1, &bc);
  }
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
    for (int s = 0; s < 2; ++s) q += (long long)P.ph.sp[s].qsign * (long long)(bc.hits[s][0] + bc.hits[s][1]);
    if (q) atomicAdd(reinterpret_cast<unsigned long long*>(&g->wall_charge), (unsigned long long)q);
    unsigned ion_lost = bc.hits[1][0] + bc.hits[1][1];
    if (ion_lost) atomicAdd(&g->src_K, (unsigned long long)ion_lost);
  }
}

__global__ void __launch_bounds__(256) k_source64(const StepParams64 P) {
  const Phys& ph = P.ph;
  const unsigned long long K = P.ctl->src_K;
  const unsigned long long n0 = P.ctl->n_cur[0], n1 = P.ctl->n_cur[1];
  __shared__ unsigned int added[2];
  if (threadIdx.x < 2) added[threadIdx.x] = 0u;
  __syncthreads();
  for (unsigned long long k = threadIdx.x; k < K; k += blockDim.x) {
    unsigned long long ide = (1ull << 63) | ((P.step & 0x7FFFFFFFull) << 32) | (2ull * k);
    uint4 w = draw4(ide, ph.seed, P.step, CH_SOURCE, 0u);
    double x = ph.src_x1_d * u01d(w.x);
    {
      uint4 u = draw4(ide, ph.seed, P.step, CH_SOURCE, 1u);
      double a0, a1, a2, a3;
      box_muller_d(u.x, u.y, a0, a1);
      box_muller_d(u.z, u.w, a2, a3);
      double v[3] = {ph.sp[0].vt_d * a0, ph.sp[0].vt_d * a1, ph.sp[0].vt_d * a2};
      if (append64<0>(P, n0, x, v, ide)) {
        deposit64<0>(P, x);
        atomicAdd(&added[0], 1u);
      }
    }
    {
      uint4 u = draw4(ide + 1ull, ph.seed, P.step, CH_SOURCE, 1u);
      double a0, a1, a2, a3;
      box_muller_d(u.x, u.y, a0, a1);
      box_muller_d(u.z, u.w, a2, a3);
      double v[3] = {ph.sp[1].vt_d * a0, ph.sp[1].vt_d * a1, ph.sp[1].vt_d * a2};
      if (append64<1>(P, n1, x, v, ide + 1ull)) {
        deposit64<1>(P, x);
        atomicAdd(&added[1], 1u);
      }
    }
  }
  __syncthreads();
  if (threadIdx.x < 2 && added[threadIdx.x]) atomicAdd(&P.ctl->n_live[threadIdx.x], (unsigned long long)added[threadIdx.x]);
  if (threadIdx.x == 0) P.ctl->source_pairs += K;
}

}  // namespace

int occupancy_step64() {
  int b = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_step64, 256, 0) != cudaSuccess || b < 1) b = 1;
  return b;
}

cudaError_t launch_step64(const StepParams64& p, int grid, cudaStream_t st) {
  k_step64<<<grid, 256, 0, st>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_source64(const StepParams64& p, cudaStream_t st) {
  k_source64<<<1, 256, 0, st>>>(p);
  return cudaGetLastError();
}
