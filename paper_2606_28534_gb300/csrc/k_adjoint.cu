// k_adjoint.cu -- kernels of the adjoint (reverse-mode gradient) of the collisionless PIC step.
//
// The forward model is the step of Sec. 2 with collisions off (gather -> Boris push -> walls ->
// deposit -> field solve), FP32 particles, signed int64 fixed-point deposit, FP64 field.  The
// absorption schedule is an input of the differentiated map: a recording run absorbs a particle at
// the first step its position leaves [0, N) and stores that step; replaying and recomputing runs
// absorb it at that step, and until then a particle standing outside [0, N) keeps the linear
// extension of its boundary cell's CIC weights (cell clamped to [0, N-1], fraction outside [0, 1)).
// Observables: J_flux = sum_n dt sum_{electrons alive after n} w v_x S(x - (N - 1)),
// S(d) = max(0, 1 - |d|), and J_fe = final field energy; parameters: V_L (uniform field
// (V_L - V_R)/(N dx) in every solve) and T_e (v = sqrt(T_e/m) xi at the load).
//
// The reverse sweep keeps, per particle, lambda = dJ/d(x, v) in FP64 and, per node, mu = dJ/dE in
// FP64.  Step n backwards (x in cell units, c/f the CIC cell and fraction):
//   rho_bar = G^T mu^{n+1}: psi = D^T mu (k_adj_field_t), chi = A^{-1} psi (the same Green's-function
//     solve as the forward, walls at 0), g_j = rho_bar_j / vol_j = dx chi_j inside, -mu_0 and mu_N
//     at the walls; dJ/dV_L += sum_j mu_j / (N dx)
//   per particle alive after n (k_adj_reverse): lambda_x += q w (g_{c'+1} - g_{c'}) [deposit of
//     x^{n+1}], the J_flux terms, lambda_vx += lambda_x dt/dx, e_bar = h [(M+I)^T lambda_v]_x,
//     lambda_x += e_bar (E_{c+1} - E_c), mu^n_c += e_bar (1 - f), mu^n_{c+1} += e_bar f,
//     lambda_v = M^T lambda_v
// and dJ/dT_e = sum over electrons of lambda_v . v^0 / (2 T_e) at the end.
#include "pic_internal.cuh"

namespace {

__device__ __forceinline__ unsigned long long to_u64(long long v) { return (unsigned long long)v; }

// The FP32 push of the adjoint model with every rounding spelled out: a replay or a recompute
// repeats the recording run bit for bit.  Returns the new (unclamped) cell.
__device__ __forceinline__ int adj_push(const AdjStep& P, int s, int c, float& f, float& vx, float& vy, float& vz) {
  float e = 0.f;
  if (P.field_mode == 0u) {
    const float E0 = (float)P.E[c], E1 = (float)P.E[c + 1];
    e = __fadd_rn(__fmul_rn(__fsub_rn(1.f, f), E0), __fmul_rn(f, E1));
  } else if (P.field_mode == 1u) {
    e = P.E_ext;
  }
  const float a = __fmul_rn(P.qmdt2[s], e);
  float mx = __fadd_rn(vx, a), my = vy, mz = vz;
  if (P.has_B) {
    const float* t = P.t[s];
    const float* q = P.s[s];
    const float px = __fadd_rn(mx, __fsub_rn(__fmul_rn(my, t[2]), __fmul_rn(mz, t[1])));
    const float py = __fadd_rn(my, __fsub_rn(__fmul_rn(mz, t[0]), __fmul_rn(mx, t[2])));
    const float pz = __fadd_rn(mz, __fsub_rn(__fmul_rn(mx, t[1]), __fmul_rn(my, t[0])));
    const float nx = __fadd_rn(mx, __fsub_rn(__fmul_rn(py, q[2]), __fmul_rn(pz, q[1])));
    const float ny = __fadd_rn(my, __fsub_rn(__fmul_rn(pz, q[0]), __fmul_rn(px, q[2])));
    const float nz = __fadd_rn(mz, __fsub_rn(__fmul_rn(px, q[1]), __fmul_rn(py, q[0])));
    mx = nx;
    my = ny;
    mz = nz;
  }
  vx = __fadd_rn(mx, a);
  vy = my;
  vz = mz;
  const float fn = __fadd_rn(f, __fmul_rn(vx, P.dtdx));
  const float fl = floorf(fn);
  int cn = c + (int)fl;
  f = __fsub_rn(fn, fl);
  if (f >= 1.f) {
    f = 0.f;
    cn += 1;
  }
  return cn;
}

// Signed fixed-point CIC deposit: W_r = rint(f 2^32), W_l = 2^32 - W_r (f may lie outside [0, 1)
// in a boundary cell of a replayed run).
__device__ __forceinline__ void adj_deposit(unsigned long long* R, int c, float f) {
  const long long wr = __double2ll_rn((double)f * 4294967296.0);
  atomicAdd(R + c, to_u64(4294967296ll - wr));
  atomicAdd(R + c + 1, to_u64(wr));
}

// One forward step of every particle (mode 0: record, 1: replay, 2: recompute into the tape).
// A CTA takes a contiguous range of particles (in load order, so a few neighbouring cells).  When
// the grid is small (priv), its deposits go to a copy of both species' node arrays in shared memory
// and only the nodes it touched are added to global memory: the integer sums are exact in any order,
// and the same-address global atomics of neighbouring particles disappear.
__global__ void __launch_bounds__(256) k_adj_push(const AdjStep P, int priv) {
  extern __shared__ unsigned long long sR[];  // priv: R_0 then R_1 of this CTA, N + 1 nodes each
  double jf = 0.0;  // this thread's J_flux terms
  const long long n = P.step;
  const int M = P.N + 1;
  const bool deposit = P.mode != 2;
  if (priv && deposit) {
    for (int j = threadIdx.x; j < 2 * M; j += blockDim.x) sR[j] = 0ull;
    __syncthreads();
  }
  const unsigned long long per = ((P.np + gridDim.x - 1) / gridDim.x + blockDim.x - 1) / blockDim.x * blockDim.x;
  const unsigned long long p_end = min(P.np, (unsigned long long)(blockIdx.x + 1) * per);
  for (unsigned long long p = (unsigned long long)blockIdx.x * per + threadIdx.x; p < p_end; p += blockDim.x) {
    const int ab = P.absorb[p];
    if (ab < n) continue;  // absorbed in an earlier step
    const int s = p < P.n0 ? 0 : 1;
    int c = P.src.cell[p];
    float f = P.src.frac[p], vx = P.src.vx[p], vy = P.src.vy[p], vz = P.src.vz[p];
    bool alive = true;
    if (!((P.frozen_mask >> s) & 1u)) {
      int cn = adj_push(P, s, c, f, vx, vy, vz);
      if (P.mode == 0) {
        if (cn < 0 || cn >= P.N) {
          P.absorb[p] = (int)n;
          alive = false;
        }
      } else {
        alive = ab > n;
        if (cn < 0) {  // linear extension of the boundary cell
          f = __fadd_rn((float)cn, f);
          cn = 0;
        } else if (cn > P.N - 1) {
          f = __fadd_rn((float)(cn - (P.N - 1)), f);
          cn = P.N - 1;
        }
      }
      c = cn;
    } else if (P.mode != 0) {
      alive = ab > n;
    }
    P.dst.cell[p] = c;
    P.dst.frac[p] = f;
    P.dst.vx[p] = vx;
    P.dst.vy[p] = vy;
    P.dst.vz[p] = vz;
    if (!alive || P.mode == 2) continue;
    adj_deposit(priv ? sR + (size_t)s * M : P.R[s], c, f);
    if (s == 0) {
      const double d = (double)(c - (P.N - 1)) + (double)f;
      const double ad = fabs(d);
      if (ad < 1.0) jf += P.flux_dtw * (double)vx * (1.0 - ad);
    }
  }
  if (P.mode == 2) return;
  if (priv) {  // the nodes this CTA deposited to
    __syncthreads();
    for (int j = threadIdx.x; j < 2 * M; j += blockDim.x) {
      const unsigned long long v = sR[j];
      if (v) atomicAdd(P.R[j >= M ? 1 : 0] + (j >= M ? j - M : j), v);
    }
  }
  // J_flux: fixed-order warp sum, then an integer 2^-40 fixed-point reduction (order-free)
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) jf += __shfl_down_sync(0xFFFFFFFFu, jf, o);
  if ((threadIdx.x & 31) == 0 && jf != 0.0) atomicAdd(P.jflux_fx, to_u64(__double2ll_rn(jf * 1099511627776.0)));
}

// Deposit of every particle as loaded (step 0's field).
__global__ void __launch_bounds__(256) k_adj_deposit0(const AdjState S, unsigned long long n0, unsigned long long np,
                                                    unsigned long long* R0, unsigned long long* R1) {
  for (unsigned long long p = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; p < np;
       p += (unsigned long long)gridDim.x * blockDim.x)
    adj_deposit(p < n0 ? R0 : R1, S.cell[p], S.frac[p]);
}

__global__ void k_adj_fill(int* a, unsigned long long n, int v) {
  for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (unsigned long long)gridDim.x * blockDim.x)
    a[i] = v;
}

// One CTA: psi / dx^2 (the right-hand side the Green's-function solve expects) at the interior
// nodes, zero at the walls, and dJ/dV_L += sum_j mu_j / (N dx) in a fixed summation order.  FP64
// runs at a small fraction of the FP32 rate on this GPU: the divisions are products with
// reciprocals formed once on the host.
__global__ void __launch_bounds__(1024) k_adj_field_t(const double* __restrict__ mu, double* __restrict__ rhs, int N,
                                                    double inv_dx, double* gV, int with_rhs,
                                                    double* __restrict__ zero_next) {
  __shared__ double part[1024];
  const int tid = threadIdx.x;
  const double half_inv_dx = 0.5 * inv_dx, inv_dx2 = inv_dx * inv_dx;
  double acc = 0.0;
  for (int j = tid; j <= N; j += 1024) {
    acc += mu[j];
    if (zero_next) zero_next[j] = 0.0;
    if (with_rhs) {
      double a = 0.0;
      if (j >= 1 && j <= N - 1) {
        if (j + 1 <= N - 1) a += mu[j + 1] * half_inv_dx;
        if (j - 1 >= 1) a -= mu[j - 1] * half_inv_dx;
        if (j == 1) a -= mu[0] * inv_dx;
        if (j == N - 1) a += mu[N] * inv_dx;
      }
      rhs[j] = a * inv_dx2;
    }
  }
  part[tid] = acc;
  __syncthreads();
  for (int o = 512; o > 0; o >>= 1) {
    if (tid < o) part[tid] += part[tid + o];
    __syncthreads();
  }
  if (tid == 0) *gV += part[0] * (inv_dx / (double)N);
}

// One backward step of every particle alive after step n.  Particles stay near their load order
// (cell order), so the lanes of a warp form runs of equal cells: the mu contributions are summed
// over each run by a segmented warp scan and the run's last lane adds them with one atomic pair.
__global__ void __launch_bounds__(256) k_adj_reverse(const AdjRev P) {
  const long long n = P.step;
  const int N = P.N;
  const int lane = threadIdx.x & 31;
  const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
  for (unsigned long long base = (unsigned long long)blockIdx.x * blockDim.x + (threadIdx.x & ~31u); base < P.np;
       base += stride) {
    const unsigned long long p = base + lane;
    int key = -1;  // the cell whose two nodes receive this lane's mu contribution (-1: none)
    double m0 = 0.0, m1 = 0.0;
    if (p < P.np && P.absorb[p] > n) {  // alive after step n (otherwise nothing depends on its state)
    const int s = p < P.n0 ? 0 : 1;
    double lx = P.lx[p], lvx = P.lvx[p], lvy = P.lvy[p], lvz = P.lvz[p];
    // deposit of x^{n+1}
    const int c1 = P.s1.cell[p];
    const float f1 = P.s1.frac[p];
    const double g0 = c1 == 0 ? -P.mu[0] : P.dx * P.chi[c1];
    const double g1 = c1 + 1 == N ? P.mu[N] : P.dx * P.chi[c1 + 1];
    lx += P.qw[s] * (g1 - g0);
    // J_flux at step n
    if (s == 0 && P.flux_dtw != 0.0) {
      const double d = (double)(c1 - (N - 1)) + (double)f1;
      const double ad = fabs(d);
      if (ad < 1.0) {
        lx += P.flux_dtw * (double)P.s1.vx[p] * (d > 0.0 ? -1.0 : (d < 0.0 ? 1.0 : 0.0));
        lvx += P.flux_dtw * (1.0 - ad);
      }
    }
    if (!((P.frozen_mask >> s) & 1u)) {
      // x^{n+1} = x^n + v_x^{n+1} dt / dx
      lvx += lx * P.dtdx;
      // v^{n+1} = M v^n + (M + I) h e(x^n)
      const double* M = P.M[s];  // row-major
      if (P.field_mode == 0u) {
        const double eb = P.h[s] * ((M[0] + 1.0) * lvx + M[3] * lvy + M[6] * lvz);
        const int c0 = P.s0.cell[p];
        const double f0 = (double)P.s0.frac[p];
        const double E0 = (double)(float)P.E[c0], E1 = (double)(float)P.E[c0 + 1];
        lx += eb * (E1 - E0);
        key = c0;
        m0 = eb * (1.0 - f0);
        m1 = eb * f0;
      }
      const double ax = M[0] * lvx + M[3] * lvy + M[6] * lvz;
      const double ay = M[1] * lvx + M[4] * lvy + M[7] * lvz;
      const double az = M[2] * lvx + M[5] * lvy + M[8] * lvz;
      lvx = ax;
      lvy = ay;
      lvz = az;
    }
    P.lx[p] = lx;
    P.lvx[p] = lvx;
    P.lvy[p] = lvy;
    P.lvz[p] = lvz;
    }
    // mu^n_c += e_bar (1 - f), mu^n_{c+1} += e_bar f: segmented sum over runs of equal cells
    const int prev = __shfl_up_sync(0xFFFFFFFFu, key, 1);
    const unsigned heads = __ballot_sync(0xFFFFFFFFu, lane == 0 || key != prev);
    const int head = 31 - __clz(heads & (0xFFFFFFFFu >> (31 - lane)));  // first lane of my run
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const double t0 = __shfl_up_sync(0xFFFFFFFFu, m0, o), t1 = __shfl_up_sync(0xFFFFFFFFu, m1, o);
      if (lane - o >= head) {
        m0 += t0;
        m1 += t1;
      }
    }
    const bool last = lane == 31 || ((heads >> (lane + 1)) & 1u);
    if (last && key >= 0) {
      atomicAdd(P.mu_next + key, m0);
      atomicAdd(P.mu_next + key + 1, m1);
    }
  }
}

// dJ/dT_e partial sums: per CTA, sum over its electrons of lambda_v . v^0 (fixed order).
__global__ void __launch_bounds__(256) k_adj_tgrad(const AdjRev P, const AdjState S0, double* partial) {
  __shared__ double part[256];
  double acc = 0.0;
  for (unsigned long long p = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; p < P.n0;
       p += (unsigned long long)gridDim.x * blockDim.x)
    acc += P.lvx[p] * (double)S0.vx[p] + P.lvy[p] * (double)S0.vy[p] + P.lvz[p] * (double)S0.vz[p];
  part[threadIdx.x] = acc;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) part[threadIdx.x] += part[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = part[0];
}

int grid_for(unsigned long long n, int cap) {
  const unsigned long long b = (n + 255) / 256;
  return (int)(b < 1 ? 1 : (b < (unsigned long long)cap ? b : (unsigned long long)cap));
}

}  // namespace

cudaError_t launch_adj_push(const AdjStep& p, int max_grid, cudaStream_t st) {
  // both species' node arrays in shared memory when they fit in 32 KB
  const size_t smem = 2 * sizeof(unsigned long long) * (size_t)(p.N + 1);
  const int priv = p.mode != 2 && smem <= 32768 ? 1 : 0;
  k_adj_push<<<grid_for(p.np, max_grid), 256, priv ? smem : 0, st>>>(p, priv);
  return cudaGetLastError();
}

cudaError_t launch_adj_deposit0(const AdjState& s, unsigned long long n0, unsigned long long np,
                                unsigned long long* R0, unsigned long long* R1, int max_grid, cudaStream_t st) {
  k_adj_deposit0<<<grid_for(np, max_grid), 256, 0, st>>>(s, n0, np, R0, R1);
  return cudaGetLastError();
}

cudaError_t launch_adj_fill(int* a, unsigned long long n, int v, cudaStream_t st) {
  k_adj_fill<<<grid_for(n, 1024), 256, 0, st>>>(a, n, v);
  return cudaGetLastError();
}

cudaError_t launch_adj_field_t(const double* mu, double* rhs, int N, double dx, double* gV, int with_rhs,
                               double* zero_next, cudaStream_t st) {
  k_adj_field_t<<<1, 1024, 0, st>>>(mu, rhs, N, 1.0 / dx, gV, with_rhs, zero_next);
  return cudaGetLastError();
}

cudaError_t launch_adj_reverse(const AdjRev& p, int max_grid, cudaStream_t st) {
  k_adj_reverse<<<grid_for(p.np, max_grid), 256, 0, st>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_adj_tgrad(const AdjRev& p, const AdjState& s0, double* partial, int blocks, cudaStream_t st) {
  k_adj_tgrad<<<blocks, 256, 0, st>>>(p, s0, partial);
  return cudaGetLastError();
}
