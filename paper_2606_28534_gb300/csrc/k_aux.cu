// k_aux.cu -- particle load, diagnostic reductions and the Philox operation.
//
// Load (paper Sec. 2: "initialization of the simulation domain, particle load"): particle i of
// species s has id i (electrons) or 2^62 | i (ions); its position and velocity come from the
// Philox blocks (id, step 0, INIT, 0) and (id, step 0, INIT, 1), evaluated in FP64 and
// rounded once to the storage precision.  Profiles: uniform (ppc per cell, random in the cell),
// exponential (inverse CDF of exp(-x/lambda) truncated to [0, L)), quiet sine (evenly spaced,
// species 0 displaced by A sin(2 pi m x / L)).
#include "pic_internal.cuh"

namespace {

struct LoadArgs {
  unsigned long long n[2];
  int profile;
  int ppc[2];
  double scale;  // EXP lambda or QUIET_SINE amplitude
  int mode;      // QUIET_SINE mode number
};

__device__ __forceinline__ void load_one(const Phys& ph, const LoadArgs& a, int s, unsigned long long i,
                                         double& x, double v[3], unsigned long long& id) {
  const int N = ph.N;
  id = s == 0 ? i : ((1ull << 62) | i);
  if (a.profile == 0) {
    uint4 w = draw4(id, ph.seed, 0ull, CH_INIT, 0u);
    x = (double)(i / (unsigned long long)a.ppc[s]) + u01d(w.x);
  } else if (a.profile == 1) {
    uint4 w = draw4(id, ph.seed, 0ull, CH_INIT, 0u);
    x = -a.scale * log(1.0 - u01d(w.x) * (1.0 - exp(-(double)N / a.scale)));
  } else {
    double x0 = ((double)i + 0.5) * (double)N / (double)a.n[s];
    x = x0;
    if (s == 0) x = x0 + a.scale * sin(2.0 * 3.14159265358979323846 * (double)a.mode * x0 / (double)N);
  }
  if (x < 0.0) x = 0.0;
  if (x >= (double)N) x = nextafter((double)N, 0.0);
  uint4 w = draw4(id, ph.seed, 0ull, CH_INIT, 1u);
  double r0 = sqrt(-2.0 * log(1.0 - u01d(w.x))), r1 = sqrt(-2.0 * log(1.0 - u01d(w.z)));
  double s0, c0, s1, c1;
  sincospi(2.0 * u01d(w.y), &s0, &c0);
  sincospi(2.0 * u01d(w.w), &s1, &c1);
  const double vt = ph.sp[s].vt_d;
  v[0] = vt * r0 * c0;
  v[1] = vt * r0 * s0;
  v[2] = vt * r1 * c1;
}

__global__ void __launch_bounds__(256) k_load32(const StepParams32 P, const LoadArgs a) {
  const unsigned long long tot = a.n[0] + a.n[1];
  for (unsigned long long g = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; g < tot;
       g += (unsigned long long)gridDim.x * blockDim.x) {
    const int s = g < a.n[0] ? 0 : 1;
    const unsigned long long i = s ? g - a.n[0] : g;
    double x, v[3];
    unsigned long long id;
    load_one(P.ph, a, s, i, x, v, id);
    double cl = floor(x);
    int c = (int)cl;
    float f = (float)(x - cl);
    if (f >= 1.f) {
      f = 0.f;
      c += 1;
      if (c >= P.ph.N) {
        c = P.ph.N - 1;
        f = 0.99999994f;
      }
    }
    const Species32 A = s ? P.sp[1] : P.sp[0];
    A.cell[i] = created_word(P.ph, s, c, id, 0ull);  // with the particle's collision countdown
    A.frac[i] = f;
    A.vx[i] = (float)v[0];
    A.vy[i] = (float)v[1];
    A.vz[i] = (float)v[2];
    A.id[i] = id;
  }
}

__global__ void __launch_bounds__(256) k_load64(const StepParams64 P, const LoadArgs a) {
  const unsigned long long tot = a.n[0] + a.n[1];
  for (unsigned long long g = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; g < tot;
       g += (unsigned long long)gridDim.x * blockDim.x) {
    const int s = g < a.n[0] ? 0 : 1;
    const unsigned long long i = s ? g - a.n[0] : g;
    double x, v[3];
    unsigned long long id;
    load_one(P.ph, a, s, i, x, v, id);
    const Species64 A = s ? P.sp[1] : P.sp[0];
    A.x[i] = x;
    A.vx[i] = v[0];
    A.vy[i] = v[1];
    A.vz[i] = v[2];
    A.id[i] = id;
    A.nk[i] = created_pair<true>(P.ph, s, id, 0ull);
  }
}

// Plain path: countdown pairs a snapshot left undrawn (0) for a species with the null-collision
// test: drawn as at creation, at the snapshot's step.
__global__ void __launch_bounds__(256) k_fill_pairs64(unsigned* __restrict__ nk, const unsigned long long* __restrict__ id,
                                                      unsigned long long n, const Phys ph, int s,
                                                      unsigned long long step) {
  for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (unsigned long long)gridDim.x * blockDim.x)
    if (nk[i] == 0u) nk[i] = created_pair<true>(ph, s, id[i], step);
}

// Plain path: sum of 0.5 m v^2 over live particles in 2^-24 fixed point (exact integer sums,
// independent of particle order and launch shape).  The FP32 step sums its own (ke_fx32).
__device__ __forceinline__ unsigned long long warp_sum64(unsigned long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xFFFFFFFFu, v, o);
  return v;
}

// Kinetic energy of the live FP32 particles, the same 2^-24 fixed point (ke_fx32) the step sums
// when asked to: the two give the same bits.
__global__ void __launch_bounds__(256) k_diag32(const StepParams32 P) {
  const unsigned long long n0 = P.ctl->n_cur[0], n1 = P.ctl->n_cur[1];
  unsigned long long acc[2] = {0ull, 0ull};
  for (unsigned long long g = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; g < n0 + n1;
       g += (unsigned long long)gridDim.x * blockDim.x) {
    const int s = g < n0 ? 0 : 1;
    const unsigned long long i = s ? g - n0 : g;
    const Species32& A = s ? P.sp[1] : P.sp[0];
    if (A.cell[i] == PIC_DEAD_CELL) continue;
    acc[s] += ke_fx32(A.vx[i], A.vy[i], A.vz[i], P.ph.sp[s].mass);
  }
  for (int s = 0; s < 2; ++s) {
    unsigned long long t = warp_sum64(acc[s]);
    if ((threadIdx.x & 31) == 0 && t) atomicAdd(&P.ctl->ke_fx[s], t);
  }
}

__global__ void __launch_bounds__(256) k_diag64(const StepParams64 P) {
  const unsigned long long n0 = P.ctl->n_cur[0], n1 = P.ctl->n_cur[1];
  unsigned long long acc[2] = {0ull, 0ull};
  for (unsigned long long g = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; g < n0 + n1;
       g += (unsigned long long)gridDim.x * blockDim.x) {
    const int s = g < n0 ? 0 : 1;
    const unsigned long long i = s ? g - n0 : g;
    const Species64 A = s ? P.sp[1] : P.sp[0];
    if (A.x[i] < 0.0) continue;
    double vx = A.vx[i], vy = A.vy[i], vz = A.vz[i];
    double e = 0.5 * P.ph.sp[s].mass_d * (vx * vx + vy * vy + vz * vz);
    acc[s] += __double2ull_rn(e * 16777216.0);
  }
  for (int s = 0; s < 2; ++s) {
    unsigned long long t = warp_sum64(acc[s]);
    if ((threadIdx.x & 31) == 0 && t) atomicAdd(&P.ctl->ke_fx[s], t);
  }
}

// Net deposited charge (exact int64) and field energy sum_j w_j 0.5 E_j^2 dx (w = 1/2 at the walls):
// block b sums a fixed run of nodes in a fixed order and writes its partial; the host adds the
// PIC_DIAG_BLOCKS partials in block order, so the result does not depend on scheduling.
__global__ void __launch_bounds__(256) k_diag_grid(const long long* __restrict__ R0, const long long* __restrict__ R1,
                                                   int sign0, int sign1, const double* __restrict__ E, int N,
                                                   double dx, Ctl* ctl) {
  __shared__ double wsum[8];
  const int seg = (N + 1 + gridDim.x - 1) / gridDim.x;
  const int a = blockIdx.x * seg, b = min(N + 1, a + seg);
  double fe = 0.0;
  long long q = 0;
  for (int j = a + (int)threadIdx.x; j < b; j += blockDim.x) {
    const double e = E[j];
    fe += ((j == 0 || j == N) ? 0.25 : 0.5) * e * e * dx;
    q += (long long)sign0 * R0[j] + (long long)sign1 * R1[j];
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    fe += __shfl_down_sync(0xFFFFFFFFu, fe, o);
    q += __shfl_down_sync(0xFFFFFFFFu, q, o);
  }
  if ((threadIdx.x & 31) == 0) {
    wsum[threadIdx.x >> 5] = fe;
    if (q) atomicAdd(reinterpret_cast<unsigned long long*>(&ctl->netq), (unsigned long long)q);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += wsum[w];
    ctl->fe_part[blockIdx.x] = t;
  }
}

// Restore: one chunk of a snapshot's per-species arrays (uploaded as they are in the blob: cell
// words, FP64 fractions and velocities, u64 ids) converted to the FP32 layout.  The host has
// already checked cells, countdowns and fractions; a fraction that rounds up to 1 moves to the next
// cell; a countdown the blob left undrawn (0) for a species with the test is drawn as at creation,
// at the snapshot's step (species 2, the neutrals, carry none).
__global__ void __launch_bounds__(256) k_restore32(const int* __restrict__ cell, const double* __restrict__ frac,
                                                   const double* __restrict__ vx, const double* __restrict__ vy,
                                                   const double* __restrict__ vz,
                                                   const unsigned long long* __restrict__ id, unsigned long long n,
                                                   Species32 dst, unsigned long long base, const Phys ph, int s,
                                                   unsigned long long step) {
  const int N = ph.N;
  for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (unsigned long long)gridDim.x * blockDim.x) {
    int c = cell[i] & PIC_CELL_MASK;
    unsigned pair = (unsigned)cell[i] >> PIC_CELL_BITS;
    if (pair == 0u && s < 2) pair = created_pair(ph, s, id[i], step);
    float f = (float)frac[i];
    if (f >= 1.f) {
      f = 0.f;
      c += 1;
      if (c >= N) {
        c = N - 1;
        f = 0.99999994f;
      }
    }
    const unsigned long long k = base + i;
    dst.cell[k] = c | (int)(pair << PIC_CELL_BITS);
    dst.frac[k] = f;
    dst.vx[k] = (float)vx[i];
    dst.vy[k] = (float)vy[i];
    dst.vz[k] = (float)vz[i];
    dst.id[k] = id[i];
  }
}

// Particle decomposition: the live particles whose id % nparts != part leave this part (marked dead;
// the next full sort compacts them away); the live counts drop by as many.
__global__ void __launch_bounds__(256) k_keep_subset(const Species32 a0, const Species32 a1, Ctl* ctl, unsigned part,
                                                     unsigned nparts) {
  const unsigned long long n0 = ctl->n_cur[0], n1 = ctl->n_cur[1];
  unsigned long long gone[2] = {0ull, 0ull};
  for (unsigned long long g = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; g < n0 + n1;
       g += (unsigned long long)gridDim.x * blockDim.x) {
    const int s = g < n0 ? 0 : 1;
    const unsigned long long i = s ? g - n0 : g;
    const Species32& A = s ? a1 : a0;
    if (A.cell[i] == PIC_DEAD_CELL || A.id[i] % nparts == part) continue;
    A.cell[i] = PIC_DEAD_CELL;
    gone[s] += 1ull;
  }
  for (int s = 0; s < 2; ++s) {
    unsigned long long t = gone[s];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xFFFFFFFFu, t, o);
    if ((threadIdx.x & 31) == 0 && t) atomicAdd(&ctl->n_live[s], (unsigned long long)(-(long long)t));
  }
}

__global__ void __launch_bounds__(256) k_philox(const uint4* __restrict__ ctr, const uint2* __restrict__ key,
                                                uint4* __restrict__ out, size_t n) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    out[i] = philox10(ctr[i], key[i]);
}

}  // namespace

cudaError_t launch_load32(const StepParams32& p, const unsigned long long n[2], int profile, int ppc0,
                          int ppc1, double scale, int mode, cudaStream_t st) {
  LoadArgs a{{n[0], n[1]}, profile, {ppc0, ppc1}, scale, mode};
  unsigned long long tot = n[0] + n[1];
  int grid = (int)((tot + 255) / 256 < 152ull * 16 ? (tot + 255) / 256 : 152ull * 16);
  if (grid < 1) grid = 1;
  k_load32<<<grid, 256, 0, st>>>(p, a);
  return cudaGetLastError();
}

cudaError_t launch_load64(const StepParams64& p, const unsigned long long n[2], int profile, int ppc0,
                          int ppc1, double scale, int mode, cudaStream_t st) {
  LoadArgs a{{n[0], n[1]}, profile, {ppc0, ppc1}, scale, mode};
  unsigned long long tot = n[0] + n[1];
  int grid = (int)((tot + 255) / 256 < 152ull * 16 ? (tot + 255) / 256 : 152ull * 16);
  if (grid < 1) grid = 1;
  k_load64<<<grid, 256, 0, st>>>(p, a);
  return cudaGetLastError();
}

cudaError_t launch_diag32(const StepParams32& p, int grid, cudaStream_t st) {
  k_diag32<<<grid, 256, 0, st>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_diag64(const StepParams64& p, int grid, cudaStream_t st) {
  k_diag64<<<grid, 256, 0, st>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_diag_grid(const long long* R0, const long long* R1, int sign0, int sign1, const double* E, int N,
                             double dx, Ctl* ctl, cudaStream_t st) {
  k_diag_grid<<<PIC_DIAG_BLOCKS, 256, 0, st>>>(R0, R1, sign0, sign1, E, N, dx, ctl);
  return cudaGetLastError();
}

cudaError_t launch_restore32(const int* cell, const double* frac, const double* vx, const double* vy, const double* vz,
                             const unsigned long long* id, unsigned long long n, const Species32& dst,
                             unsigned long long base, const Phys& ph, int species, unsigned long long step,
                             cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  const unsigned long long blocks = (n + 255) / 256;
  const int grid = (int)(blocks < 152ull * 16 ? blocks : 152ull * 16);
  k_restore32<<<grid, 256, 0, st>>>(cell, frac, vx, vy, vz, id, n, dst, base, ph, species, step);
  return cudaGetLastError();
}

cudaError_t launch_fill_pairs64(unsigned* nk, const unsigned long long* id, unsigned long long n, const Phys& ph,
                                int species, unsigned long long step, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  const unsigned long long blocks = (n + 255) / 256;
  const int grid = (int)(blocks < 152ull * 16 ? blocks : 152ull * 16);
  k_fill_pairs64<<<grid, 256, 0, st>>>(nk, id, n, ph, species, step);
  return cudaGetLastError();
}

namespace {
__global__ void k_store_u64(unsigned long long* p, unsigned long long v) { *p = v; }

// Self-test of the bounded wait: an mbarrier that expects two arrivals and receives one never
// completes its phase; the wait gives up after its time limit and the kernel records that.  No copy
// is in flight and nothing else waits on this barrier.
__global__ void k_selftest_wait(unsigned long long* out) {
  __shared__ __align__(8) unsigned long long bar;
  if (threadIdx.x != 0) return;
  mbar_init(&bar, 2u);
  mbar_init_fence();
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&bar)) : "memory");
  const unsigned long long t0 = global_ns();
  const bool done = mbar_wait_bounded(&bar, 0u);
  out[1] = global_ns() - t0;
  out[0] = done ? 0ull : (unsigned long long)ERR_TIMEOUT;
}
}  // namespace

cudaError_t launch_selftest_wait(unsigned long long* out, cudaStream_t st) {
  k_selftest_wait<<<1, 32, 0, st>>>(out);
  return cudaGetLastError();
}

cudaError_t launch_store_u64(unsigned long long* p, unsigned long long v, cudaStream_t st) {
  k_store_u64<<<1, 1, 0, st>>>(p, v);
  return cudaGetLastError();
}

cudaError_t launch_keep_subset(const Species32& a0, const Species32& a1, Ctl* ctl, unsigned part, unsigned nparts,
                               cudaStream_t st) {
  k_keep_subset<<<152 * 8, 256, 0, st>>>(a0, a1, ctl, part, nparts);
  return cudaGetLastError();
}

cudaError_t launch_philox(const uint32_t* ctr, const uint32_t* key, uint32_t* out, size_t n, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  size_t blocks = (n + 255) / 256;
  int grid = (int)(blocks < 152 * 32 ? blocks : 152 * 32);
  k_philox<<<grid, 256, 0, st>>>(reinterpret_cast<const uint4*>(ctr), reinterpret_cast<const uint2*>(key),
                                 reinterpret_cast<uint4*>(out), n);
  return cudaGetLastError();
}
