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
    A.cell[i] = c;
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
  }
}

// Sum of 0.5 m v^2 over live particles in 2^-24 fixed point: exact integer sums, independent of
// particle order and of the launch shape.
__device__ __forceinline__ unsigned long long warp_sum64(unsigned long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xFFFFFFFFu, v, o);
  return v;
}

__global__ void __launch_bounds__(256) k_diag32(const StepParams32 P) {
  const unsigned long long n0 = P.ctl->n_cur[0], n1 = P.ctl->n_cur[1];
  unsigned long long acc[2] = {0ull, 0ull};
  for (unsigned long long g = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; g < n0 + n1;
       g += (unsigned long long)gridDim.x * blockDim.x) {
    const int s = g < n0 ? 0 : 1;
    const unsigned long long i = s ? g - n0 : g;
    const Species32 A = s ? P.sp[1] : P.sp[0];
    if (A.cell[i] == PIC_DEAD_CELL) continue;
    double vx = A.vx[i], vy = A.vy[i], vz = A.vz[i];
    double e = 0.5 * P.ph.sp[s].mass_d * (vx * vx + vy * vy + vz * vz);
    acc[s] += __double2ull_rn(e * 16777216.0);
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

cudaError_t launch_philox(const uint32_t* ctr, const uint32_t* key, uint32_t* out, size_t n, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  size_t blocks = (n + 255) / 256;
  int grid = (int)(blocks < 152 * 32 ? blocks : 152 * 32);
  k_philox<<<grid, 256, 0, st>>>(reinterpret_cast<const uint4*>(ctr), reinterpret_cast<const uint2*>(key),
                                 reinterpret_cast<uint4*>(out), n);
  return cudaGetLastError();
}
